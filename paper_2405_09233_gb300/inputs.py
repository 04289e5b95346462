"""Seeded synthetic workloads for the Sylvester tensor equation A*X - X*B = C.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no T-product, no FFT, no solve).  Both the CUDA path and
the CPU oracle take their inputs from here, so the two see identical bytes.

Tensors are numpy arrays of shape (n1, n2, p) indexed [i, j, k] as in the
paper's MATLAB notation (frontal slice k is X[:, :, k]).  The device layout is
column-major, X(i, j, k) at i + n1*(j + n2*k); `to_device_layout` returns that
order as a C-contiguous array of shape (p, n2, n1).

Workloads (the paper's own experiment uses convection-diffusion slices with an
unstated viscosity and an unseeded right-hand side, so these synthetic
families stand in for it):

* dense family: A^(1) = tridiag(-1, 4, -1) + g*G/sqrt(n), A^(k>=2) = g*G/sqrt(n);
  B^(1) = -tridiag(-1, 4, -1) + g*G'/sqrt(s), B^(k>=2) = g*G'/sqrt(s);
  every slice draws a fresh i.i.d. N(0,1) matrix; g = 0.1 (0.3 for the
  mixed-precision family); X* entries i.i.d. U(-1, 1); C = M(X*).
* sparse family: A^(1) = 5-point Laplacian on a g x g grid (4 on the diagonal,
  -1 for each N/S/E/W neighbour, Dirichlet), A^(2..p) with 4 distinct random
  off-diagonal columns per row and N(0, 0.05^2) values; B dense with
  B^(1) = -4 I + 0.1 G'/sqrt(s) and B^(k>=2) = 0.1 G'/sqrt(s).
* batched family: many dense-family instances with n log-uniform in
  [64, 1024], s uniform in [16, 128], p drawn from {4, 8, 16}.
* convection-diffusion family (the paper's §6 example, with the viscosity mu
  given explicitly and a seeded right-hand side): A^(i) = mu/h1^2 tridiag(-1, 2, -1)
  + a_i/(4 h1) T_n and B^(i) = mu/h2^2 tridiag(-1, 2, -1) + b_i/(4 h2) T_s, with
  T the banded matrix of 3 on the diagonal, -5 above it, 1 two above it and 1 below
  it, a_i = i, b_i = p + i, h1 = 1/(n+1), h2 = 1/(s+1); C entries i.i.d. U(0, 1).
"""
from __future__ import annotations

import dataclasses
import numpy as np


def to_device_layout(X: np.ndarray) -> np.ndarray:
    """(n1, n2, p) tensor -> C-contiguous (p, n2, n1) array with the same bytes as column-major X."""
    return np.ascontiguousarray(np.asarray(X).transpose(2, 1, 0))


def from_device_layout(Y: np.ndarray) -> np.ndarray:
    """Inverse of `to_device_layout`: (p, n2, n1) array -> (n1, n2, p) tensor view."""
    return np.asarray(Y).transpose(2, 1, 0)


def tridiag(n: int, lo: float, d: float, up: float) -> np.ndarray:
    T = np.zeros((n, n))
    idx = np.arange(n)
    T[idx, idx] = d
    T[idx[1:], idx[:-1]] = lo
    T[idx[:-1], idx[1:]] = up
    return T


@dataclasses.dataclass
class DenseProblem:
    A: np.ndarray      # (n, n, p)
    B: np.ndarray      # (s, s, p)
    Xstar: np.ndarray  # (n, s, p), the manufactured solution
    seed: int
    scale: float

    @property
    def shape(self):
        n, s, p = self.Xstar.shape
        return n, s, p


def dense_problem(n: int, s: int, p: int, seed: int, scale: float = 0.1) -> DenseProblem:
    """Dense family.  Draw order: G for A slices 1..p, then G' for B slices 1..p, then X*."""
    rng = np.random.default_rng(seed)
    A = np.empty((n, n, p), order="F")
    for k in range(p):
        A[:, :, k] = (scale / np.sqrt(n)) * rng.standard_normal((n, n))
    A[:, :, 0] += tridiag(n, -1.0, 4.0, -1.0)
    B = np.empty((s, s, p), order="F")
    for k in range(p):
        B[:, :, k] = (scale / np.sqrt(s)) * rng.standard_normal((s, s))
    B[:, :, 0] -= tridiag(s, -1.0, 4.0, -1.0)
    Xstar = np.asfortranarray(rng.uniform(-1.0, 1.0, size=(n, s, p)))
    return DenseProblem(A, B, Xstar, seed, scale)


def random_tensor(shape, seed: int, dist: str = "normal") -> np.ndarray:
    rng = np.random.default_rng(seed)
    if dist == "normal":
        return np.asfortranarray(rng.standard_normal(shape))
    return np.asfortranarray(rng.uniform(-1.0, 1.0, size=shape))


@dataclasses.dataclass
class CsrSlice:
    rowptr: np.ndarray  # int32 (n+1,)
    col: np.ndarray     # int32 (nnz,)
    val: np.ndarray     # float64 (nnz,)

    def to_dense(self, n: int) -> np.ndarray:
        D = np.zeros((n, n))
        for i in range(n):
            for q in range(self.rowptr[i], self.rowptr[i + 1]):
                D[i, self.col[q]] += self.val[q]
        return D


@dataclasses.dataclass
class SparseProblem:
    slices: list          # p CsrSlice objects, A^(1..p)
    n: int
    B: np.ndarray         # (s, s, p)
    Xstar: np.ndarray     # (n, s, p)
    seed: int

    @property
    def p(self):
        return len(self.slices)

    def dense_A(self) -> np.ndarray:
        A = np.zeros((self.n, self.n, self.p), order="F")
        for k, sl in enumerate(self.slices):
            A[:, :, k] = sl.to_dense(self.n)
        return A


def laplacian_5pt(g: int) -> CsrSlice:
    """Unscaled 5-point stencil on a g x g grid, rows in lexicographic (x fastest) order."""
    n = g * g
    rowptr = np.zeros(n + 1, dtype=np.int32)
    cols, vals = [], []
    for r in range(n):
        x, y = r % g, r // g
        entries = []
        if y > 0:
            entries.append((r - g, -1.0))
        if x > 0:
            entries.append((r - 1, -1.0))
        entries.append((r, 4.0))
        if x < g - 1:
            entries.append((r + 1, -1.0))
        if y < g - 1:
            entries.append((r + g, -1.0))
        for c, v in entries:
            cols.append(c)
            vals.append(v)
        rowptr[r + 1] = len(cols)
    return CsrSlice(rowptr, np.asarray(cols, dtype=np.int32), np.asarray(vals))


def random_sparse_slice(n: int, nnz_per_row: int, sigma: float, rng) -> CsrSlice:
    """nnz_per_row distinct off-diagonal columns per row (sorted), values N(0, sigma^2)."""
    rowptr = np.arange(0, n * nnz_per_row + 1, nnz_per_row, dtype=np.int32)
    col = np.empty(n * nnz_per_row, dtype=np.int32)
    for i in range(n):
        c = rng.choice(n - 1, size=nnz_per_row, replace=False)
        c = np.where(c >= i, c + 1, c)  # skip the diagonal
        col[i * nnz_per_row:(i + 1) * nnz_per_row] = np.sort(c)
    val = sigma * rng.standard_normal(n * nnz_per_row)
    return CsrSlice(rowptr, col, val)


def sparse_problem(grid: int, s: int, p: int, seed: int, nnz_per_row: int = 4,
                   sigma: float = 0.05) -> SparseProblem:
    """Sparse family.  Draw order: slices 2..p (pattern then values), then B, then X*."""
    rng = np.random.default_rng(seed)
    n = grid * grid
    slices = [laplacian_5pt(grid)]
    for _ in range(1, p):
        slices.append(random_sparse_slice(n, nnz_per_row, sigma, rng))
    B = np.empty((s, s, p), order="F")
    for k in range(p):
        B[:, :, k] = (0.1 / np.sqrt(s)) * rng.standard_normal((s, s))
    B[:, :, 0] -= 4.0 * np.eye(s)
    Xstar = np.asfortranarray(rng.uniform(-1.0, 1.0, size=(n, s, p)))
    return SparseProblem(slices, n, B, Xstar, seed)


@dataclasses.dataclass
class BatchedSpec:
    n: int
    s: int
    p: int
    seed: int
    tol: float


def batched_specs(count: int, seed: int, mixed_tol: bool = False,
                  n_range=(64, 1024), s_range=(16, 128), p_choices=(4, 8, 16)):
    """Instance shapes for the batched family; instance i uses seed `seed*1000 + i`."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        s = int(rng.integers(s_range[0], s_range[1] + 1))
        p = int(rng.choice(np.asarray(p_choices)))
        tol = float(10.0 ** rng.uniform(-10.0, -8.0)) if mixed_tol else 1e-10
        specs.append(BatchedSpec(n, s, p, seed * 1000 + i, tol))
    return specs


# Named workloads with their sizes.
WORKLOADS = {
    "dense_n24_s24_p4": dict(n=24, s=24, p=4, scale=0.1, restart=20),
    "dense_n1024_s1024_p16": dict(n=1024, s=1024, p=16, scale=0.1, restart=30),
    "dense_n4096_s256_p32_g0.3": dict(n=4096, s=256, p=32, scale=0.3, restart=40),
    "sparse_lap128_s32_p8": dict(grid=128, s=32, p=8),
    "batched_256": dict(count=256),
}


def convection_band(n: int) -> np.ndarray:
    """The banded n x n matrix of the paper's convection term: 1 below the diagonal, 3 on it, -5 above it
    and 1 two above it."""
    T = np.zeros((n, n))
    i = np.arange(n)
    T[i, i] = 3.0
    T[i[1:], i[:-1]] = 1.0
    T[i[:-1], i[1:]] = -5.0
    T[i[:-2], i[2:]] = 1.0
    return T


@dataclasses.dataclass
class ConvDiffProblem:
    A: np.ndarray          # n x n x p
    B: np.ndarray          # s x s x p
    C: np.ndarray          # n x s x p, entries U(0, 1)
    mu: float
    seed: int


def convdiff_problem(n: int, s: int, p: int, mu: float, seed: int) -> ConvDiffProblem:
    """The convection-diffusion family of the paper's §6 example (frontal slices i = 1..p)."""
    h1, h2 = 1.0 / (n + 1), 1.0 / (s + 1)
    A = np.empty((n, n, p), order="F")
    B = np.empty((s, s, p), order="F")
    Ln, Ls = tridiag(n, -1.0, 2.0, -1.0), tridiag(s, -1.0, 2.0, -1.0)
    Tn, Ts = convection_band(n), convection_band(s)
    for i in range(1, p + 1):
        A[:, :, i - 1] = (mu / h1 ** 2) * Ln + (i / (4 * h1)) * Tn
        B[:, :, i - 1] = (mu / h2 ** 2) * Ls + ((p + i) / (4 * h2)) * Ts
    rng = np.random.default_rng(seed)
    C = np.asfortranarray(rng.uniform(0.0, 1.0, size=(n, s, p)))
    return ConvDiffProblem(A, B, C, mu, seed)
