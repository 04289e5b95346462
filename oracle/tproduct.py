"""T-product algebra of §2, from the definitions.  Oracle: test infrastructure only.

Tensors are float64 numpy arrays of shape (n1, n2, p), indexed [i, j, k] like
the paper's MATLAB notation; A[:, :, k] is the frontal slice A^(k+1).
"""
from __future__ import annotations

import numpy as np

# Above this many entries in bcirc(A) the T-product is evaluated block row by
# block row (the same sum as the materialised product, without storing bcirc).
_BCIRC_MATERIALISE_LIMIT = 4_000_000


def bcirc(A: np.ndarray) -> np.ndarray:
    """Block-circulant matrix of §2.1: block (r, c) is the frontal slice A^((r - c) mod p)."""
    n1, n2, p = A.shape
    M = np.zeros((n1 * p, n2 * p), dtype=A.dtype)
    for r in range(p):
        for c in range(p):
            M[r * n1:(r + 1) * n1, c * n2:(c + 1) * n2] = A[:, :, (r - c) % p]
    return M


def unfold(B: np.ndarray) -> np.ndarray:
    """§2.1: frontal slices stacked vertically, (n2*p) x m."""
    p = B.shape[2]
    return np.concatenate([B[:, :, k] for k in range(p)], axis=0)


def fold(M: np.ndarray, p: int) -> np.ndarray:
    """§2.1: inverse of unfold."""
    n = M.shape[0] // p
    return np.stack([M[k * n:(k + 1) * n, :] for k in range(p)], axis=2)


def tprod_bcirc(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Definition 2.1 verbatim: A*B = fold(bcirc(A) unfold(B))."""
    assert A.shape[1] == B.shape[0] and A.shape[2] == B.shape[2]
    return fold(bcirc(A) @ unfold(B), A.shape[2])


def tprod_blockrow(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Definition 2.1 evaluated one block row of bcirc(A) at a time.

    Block row k of bcirc(A) times unfold(B) is sum_c A^((k - c) mod p) B^(c),
    so this is the same sum as `tprod_bcirc`, in the same order of blocks.
    """
    assert A.shape[1] == B.shape[0] and A.shape[2] == B.shape[2]
    n1, _, p = A.shape
    m = B.shape[1]
    dt = np.result_type(A, B)
    C = np.zeros((n1, m, p), dtype=dt)
    for k in range(p):
        acc = np.zeros((n1, m), dtype=dt)
        for c in range(p):
            acc += A[:, :, (k - c) % p] @ B[:, :, c]
        C[:, :, k] = acc
    return C


def tprod(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """T-product (Definition 2.1); materialises bcirc(A) when it is small."""
    n1, n2, p = A.shape
    if n1 * n2 * p * p <= _BCIRC_MATERIALISE_LIMIT:
        return tprod_bcirc(A, B)
    return tprod_blockrow(A, B)


def tentry(A: np.ndarray, B: np.ndarray, i: int, j: int, k: int) -> float:
    """One entry (A*B)(i, j, k) of Definition 2.1: row i of block row k of bcirc(A) times column j of unfold(B)."""
    p = A.shape[2]
    return float(sum(A[i, :, (k - c) % p] @ B[:, j, c] for c in range(p)))


def ttranspose(A: np.ndarray) -> np.ndarray:
    """Definition 2.2(4): transpose each frontal slice, then reverse the order of slices 2..p."""
    n1, n2, p = A.shape
    T = np.zeros((n2, n1, p), dtype=A.dtype)
    T[:, :, 0] = A[:, :, 0].T
    for k in range(1, p):
        T[:, :, k] = A[:, :, p - k].T
    return T


def identity(n: int, p: int) -> np.ndarray:
    """Definition 2.2(1): first frontal slice I_n, the others zero."""
    I = np.zeros((n, n, p))
    I[:, :, 0] = np.eye(n)
    return I


def tube_e(p: int) -> np.ndarray:
    """The unit tube e (1 x 1 x p) with unfold(e) = (1, 0, ..., 0)^T."""
    e = np.zeros((1, 1, p))
    e[0, 0, 0] = 1.0
    return e


def inner(A: np.ndarray, B: np.ndarray) -> float:
    """Definition 2.3: <A, B> = sum of a_ijk b_ijk (real tensors)."""
    return float(np.sum(A * B))


def cttranspose(A: np.ndarray) -> np.ndarray:
    """Conjugate of the Definition 2.2(4) transpose; for a real tensor it is the transpose itself.

    Its Fourier slices are the conjugate transposes of those of A, which is what
    the orthogonality U^T * U = I of §4 means once U has complex entries.
    """
    return np.conj(ttranspose(A))


def norm(A: np.ndarray) -> float:
    """Definition 2.3: ||A||_F = sqrt(<A, A>)."""
    return float(np.sqrt(inner(A, A)))


def tdiamond(As, Bs) -> np.ndarray:
    """T-diamond product of §2: the matrix of inner products <A_i, B_j>."""
    return np.array([[inner(a, b) for b in Bs] for a in As])


def dft_matrix(p: int) -> np.ndarray:
    """The DFT matrix F_p, F[k, t] = exp(-2 pi i k t / p) (MATLAB fft convention, unnormalised)."""
    kt = np.outer(np.arange(p), np.arange(p)) % p
    return np.exp(-2j * np.pi * kt / p)


def dft3(A: np.ndarray) -> np.ndarray:
    """DFT of every mode-3 tube by the explicit DFT matrix (§2, `fft(A, [], 3)`)."""
    return np.einsum("ijt,kt->ijk", A.astype(complex), dft_matrix(A.shape[2]))


def idft3(Ah: np.ndarray) -> np.ndarray:
    """Inverse of dft3 (`ifft(., [], 3)`, with the 1/p factor)."""
    p = Ah.shape[2]
    return np.einsum("ijk,tk->ijt", Ah, np.conj(dft_matrix(p))) / p


def tube_inverse(z: np.ndarray) -> np.ndarray:
    """Definition 2.2(2): the tube z^{-1} with z*z^{-1} = e, through its Fourier coefficients."""
    zh = dft3(z.reshape(1, 1, -1))
    if np.any(np.abs(zh) == 0):
        raise ZeroDivisionError("tube is not invertible (a Fourier coefficient is zero)")
    zinv = idft3(1.0 / zh).reshape(z.shape)
    return np.real(zinv) if np.isrealobj(z) else zinv
