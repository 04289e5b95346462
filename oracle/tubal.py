"""Normalize, Tubal-QR, Tubal Block Arnoldi and TBAS(m) (§5).  Oracle: test infrastructure only.

Readings of the paper taken here:
  * Normalization1 (cited from Kilmer et al., not restated in the paper):
    v = u * a with u^T * u = e.  Per Fourier index k of the DFT along mode 3,
    a_k = ||v_k||_2 and u_k = v_k / a_k; u and a are the inverse DFTs.  A
    Fourier slice is numerically zero when a_k <= 1e-12 * ref, with ref the
    largest a_k of v itself.  Then a_k = 0 and u_k = e_1 (first unit vector),
    which keeps u^T * u = e.
  * Inside Tubal-QR (Algorithm 6) Normalize is applied to a column after it
    was orthogonalised against the previous ones.  There the scale ref is the
    largest Fourier-slice norm of the column *before* orthogonalisation, so a
    column that depends on the previous ones (whose orthogonalised remainder
    is rounding noise) counts as rank deficient instead of having its noise
    normalised.  The unit vector of a rank-deficient slice is then chosen
    orthogonal to the previous columns of that slice, so that Q^T * Q = I as
    Theorem 5.1 states: the first e_i (i = 1, 2, ...) whose component
    orthogonal to them has squared norm >= 1/(2n), orthogonalised (twice)
    and normalised.  Some e_i always qualifies: the squared norms of those
    components sum to n - j >= 1 over the n unit vectors.
  * Algorithm 6's inner loop runs over i = 1..j-1 (the printed "i = 2..j-1"
    and the double normalisation of the first column are read as slips).
  * Tubal Block Arnoldi applies A, not M, in its loop (the paper's claim that
    both give the same block Krylov space); M is used for R0 and the true
    residual.  The TBAS projected equation is H_m*Y - Y*B = C1 with
    C1 = V_m^T * R0, solved by t-Bartels-Stewart (Algorithm 5).
  * TBAS(m) tests the true residual after each cycle, relative to ||C||_F.
  * Block breakdown (the new block W is ~0 after orthogonalisation, i.e. the
    block Krylov space is invariant) stops the Arnoldi loop early; a rank
    deficient but nonzero block is only handled by the Normalize tie-break.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional

import numpy as np

from .tproduct import dft3, idft3, tprod, ttranspose, norm
from .schur import t_bartels_stewart

NORMALIZE_TINY = 1e-12
BLOCK_BREAKDOWN_REL = 1e-13


def fourier_norms(v: np.ndarray) -> np.ndarray:
    """a_k = ||v_k||_2 for every Fourier index k of a lateral slice v (n x 1 x p)."""
    return np.linalg.norm(dft3(v)[:, 0, :], axis=0)


def completion_vector(P: np.ndarray) -> np.ndarray:
    """A unit vector orthogonal to the orthonormal columns of P (n x j, complex, j < n): the first
    e_i whose component orthogonal to them has squared norm >= 1/(2n), orthogonalised twice."""
    n = P.shape[0]
    for i in range(n):
        z = np.zeros(n, dtype=complex)
        z[i] = 1.0
        for _ in range(2):
            z = z - P @ (np.conj(P.T) @ z)
        nz = np.linalg.norm(z)
        if nz * nz >= 1.0 / (2 * n):
            return z / nz
    raise AssertionError("no unit vector has a component orthogonal to the previous columns")


def normalize(v: np.ndarray, ref: Optional[float] = None, prev: Optional[np.ndarray] = None):
    """Normalization1: v (n x 1 x p) = u * a with u^T * u = e; returns (u, a).

    ref: the scale below which a Fourier slice counts as zero (times NORMALIZE_TINY); default the
    largest a_k of v.  prev: the columns (n x j x p) that u must be orthogonal to in a rank-deficient
    slice (Tubal-QR); default none, which gives u_k = e_1 there.
    """
    n, _, p = v.shape
    vh = dft3(v)[:, 0, :]                     # n x p Fourier coefficients
    a = np.linalg.norm(vh, axis=0)            # a_k = ||v_k||_2
    if ref is None:
        ref = a.max() if p else 0.0
    prevh = dft3(prev) if prev is not None and prev.shape[1] > 0 else None
    uh = np.zeros_like(vh)
    ah = np.zeros(p, dtype=complex)
    for k in range(p):
        if a[k] > NORMALIZE_TINY * ref:
            uh[:, k] = vh[:, k] / a[k]
            ah[k] = a[k]
        elif prevh is None:
            uh[0, k] = 1.0
        else:
            uh[:, k] = completion_vector(prevh[:, :, k])
    u = np.real(idft3(uh[:, None, :]))
    at = np.real(idft3(ah[None, None, :]))
    return u, at


def tubal_qr(Amat: np.ndarray):
    """Algorithm 6 (Tubal-QR): A = Q * R, Q^T * Q = I, R upper triangular in tubes."""
    n, m, p = Amat.shape
    Q = np.zeros((n, m, p))
    R = np.zeros((m, m, p))
    for j in range(m):
        W = Amat[:, j:j + 1, :].copy()
        ref = fourier_norms(W).max()                # scale of the column before orthogonalisation
        for i in range(j):
            Qi = Q[:, i:i + 1, :]
            rij = tprod(ttranspose(Qi), W)          # tube V_i^T * W
            R[i:i + 1, j:j + 1, :] = rij
            W = W - tprod(Qi, rij)
        q, a = normalize(W, ref=ref, prev=Q[:, :j, :])
        Q[:, j:j + 1, :] = q
        R[j:j + 1, j:j + 1, :] = a
    return Q, R


def tprod_sparse(slices, B: np.ndarray) -> np.ndarray:
    """Definition 2.1 with the frontal slices of A given as scipy sparse matrices (block-row form)."""
    p = len(slices)
    n = slices[0].shape[0]
    C = np.zeros((n, B.shape[1], p))
    for k in range(p):
        acc = np.zeros((n, B.shape[1]))
        for c in range(p):
            acc += slices[(k - c) % p] @ B[:, :, c]
        C[:, :, k] = acc
    return C


@dataclasses.dataclass
class TBAResult:
    V: list                 # V_1..V_{m+1}, each n x s x p
    H: dict                 # (i, j) -> s x s x p block, 0-based
    H0: np.ndarray          # s x s x p, R-factor of the starting block
    m: int

    def Hm(self) -> np.ndarray:
        """Block Hessenberg H_m (ms x ms x p) of §5.1."""
        s, p = self.H0.shape[0], self.H0.shape[2]
        out = np.zeros((self.m * s, self.m * s, p))
        for (i, j), blk in self.H.items():
            if i < self.m:
                out[i * s:(i + 1) * s, j * s:(j + 1) * s, :] = blk
        return out

    def Vm(self) -> np.ndarray:
        return np.concatenate(self.V[:self.m], axis=1)


def tba(applyA: Callable, V: np.ndarray, m: int) -> TBAResult:
    """Algorithm 7 (Tubal Block Arnoldi) with the operator X -> A*X given as `applyA`."""
    V1, H0 = tubal_qr(V)
    Vs = [V1]
    H = {}
    scale = norm(V)
    for j in range(m):
        W = applyA(Vs[j])
        for i in range(j + 1):
            Hij = tprod(ttranspose(Vs[i]), W)
            H[(i, j)] = Hij
            W = W - tprod(Vs[i], Hij)
        if norm(W) <= BLOCK_BREAKDOWN_REL * scale:
            # The block Krylov space is invariant: stop with j+1 blocks and a zero H_{j+2,j+1}.
            H[(j + 1, j)] = np.zeros_like(H0)
            Vs.append(np.zeros_like(V1))
            return TBAResult(Vs, H, H0, j + 1)
        Vn, Hn = tubal_qr(W)
        H[(j + 1, j)] = Hn
        Vs.append(Vn)
    return TBAResult(Vs, H, H0, m)


@dataclasses.dataclass
class TBASResult:
    X: np.ndarray
    history: list        # Proposition 5.2 estimate after each cycle
    true_res: list       # initial, then after each cycle
    cycles: int
    status: str
    normC: float

    @property
    def relres(self) -> float:
        return self.true_res[-1] / self.normC


def tbas(A, B: np.ndarray, C: np.ndarray, X0=None, m: int = 10, tol: float = 1e-10,
         max_restarts: int = 100, applyA: Optional[Callable] = None) -> TBASResult:
    """Algorithm 8, TBAS(m).  A is a dense tensor, or pass `applyA` (e.g. sparse slices)."""
    if applyA is None:
        applyA = lambda X: tprod(A, X)  # noqa: E731
    applyM = lambda X: applyA(X) - tprod(X, B)  # noqa: E731  Eq. (2)
    X = np.zeros_like(C) if X0 is None else np.array(X0, dtype=float)
    normC = norm(C)
    R = C - applyM(X)
    res = norm(R)
    hist, true_res = [], [res]
    if res <= tol * normC:
        return TBASResult(X, hist, true_res, 0, "ok", normC)
    s = C.shape[1]
    for cycle in range(max_restarts):
        arn = tba(applyA, R, m)                                 # step 3a
        Vm = arn.Vm()
        C1 = tprod(ttranspose(Vm), R)                           # V_m^T * R0
        Y = t_bartels_stewart(arn.Hm(), B, C1)                  # step 3b
        mm = arn.m
        est = norm(tprod(arn.H[(mm, mm - 1)], Y[(mm - 1) * s:, :, :]))  # Proposition 5.2
        X = X + tprod(Vm, Y)                                    # step 3c
        R = C - applyM(X)
        res = norm(R)
        hist.append(est)
        true_res.append(res)
        if res <= tol * normC:
            return TBASResult(X, hist, true_res, cycle + 1, "ok", normC)
    return TBASResult(X, hist, true_res, max_restarts, "not_converged", normC)

