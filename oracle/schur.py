"""t-Schur decomposition and t-Bartels-Stewart (§4).  Oracle: test infrastructure only.

Readings of the paper taken here:
  * The Fourier slices of a real tensor are complex, so the Schur form of
    Algorithm 4 is computed as a complex Schur form of each Fourier slice
    k = 0..floor(p/2), the slices k > p/2 being the conjugates of slices p-k
    (Theorem 4.1's "real" U and R do not exist in general).  U and R are then
    complex tensors with upper-triangular Fourier slices, and "U^T" means the
    conjugate transpose (`cttranspose`).
  * The equation solved is A*X - X*B = C (Eq. (2) form), so the triangular
    equation is R_A*Y - Y*R_B = C1 with Y = U_A^T*X*U_B, C1 = U_A^T*C*U_B.
  * t-back-substitution (Remark 4.1) treats tubes as scalars: column j of Y
    solves (R_A - r^B_jj I) y_j = c_j + sum_{i<j} y_i r^B_ij, and that upper
    triangular system is solved from the last row up, dividing by a tube with
    the tube inverse of Definition 2.2(2).
  * X is real: the result is the real part, whose imaginary residue is
    returned for checking.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .tproduct import dft3, idft3, tprod, cttranspose, tube_inverse


def t_schur(A: np.ndarray):
    """Algorithm 4: A = U * R * U^T with U orthogonal and R upper triangular (complex tensors)."""
    n, _, p = A.shape
    Ah = dft3(A)
    Uh = np.zeros((n, n, p), dtype=complex)
    Rh = np.zeros((n, n, p), dtype=complex)
    for k in range(p // 2 + 1):
        T, Z = scipy.linalg.schur(Ah[:, :, k], output="complex")
        Uh[:, :, k], Rh[:, :, k] = Z, T
        if 0 < k < p - k:
            Uh[:, :, p - k], Rh[:, :, p - k] = np.conj(Z), np.conj(T)
    return idft3(Uh), idft3(Rh)


def circulant(a: np.ndarray) -> np.ndarray:
    """Matrix of the tube product with the tube a: (a * b)[t] = sum_u a[(t - u) mod p] b[u]."""
    p = a.shape[-1]
    t = np.arange(p)
    return a[..., (t[:, None] - t[None, :]) % p]


def t_back_substitution(RA: np.ndarray, RB: np.ndarray, C1: np.ndarray) -> np.ndarray:
    """Remark 4.1: solve R_A*Y - Y*R_B = C1 for upper triangular R_A (n x n x p), R_B (s x s x p)."""
    n, s, p = C1.shape
    dt = np.result_type(RA, RB, C1)
    Y = np.zeros((n, s, p), dtype=dt)
    CA = circulant(RA)          # CA[l, q] is the p x p matrix of the tube product with RA(l, q, :)
    CB = circulant(RB)
    for j in range(s):
        rhs = C1[:, j, :].astype(dt)
        for i in range(j):      # + sum_{i<j} y_i * r^B_ij (tube products)
            rhs = rhs + np.einsum("tu,lu->lt", CB[i, j], Y[:, i, :])
        for l in range(n - 1, -1, -1):
            acc = rhs[l].copy()
            if l + 1 < n:       # - sum_{q>l} r^A_lq * y_qj
                acc -= np.einsum("qtu,qu->t", CA[l, l + 1:], Y[l + 1:, j, :])
            d = RA[l, l, :] - RB[j, j, :]
            Y[l, j, :] = circulant(tube_inverse(d.reshape(1, 1, p)).reshape(p)) @ acc
    return Y


def t_bartels_stewart(A: np.ndarray, B: np.ndarray, C: np.ndarray, return_imag: bool = False):
    """Algorithm 5 for A*X - X*B = C (A n x n x p, B s x s x p, C n x s x p)."""
    UA, RA = t_schur(A)
    UB, RB = t_schur(B)
    C1 = tprod(tprod(cttranspose(UA), C), UB)
    Y = t_back_substitution(RA, RB, C1)
    X = tprod(tprod(UA, Y), cttranspose(UB))
    if return_imag:
        return np.real(X), float(np.max(np.abs(np.imag(X))) if X.size else 0.0)
    return np.real(X)
