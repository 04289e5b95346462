"""Pins for the oracle's T-product algebra (§2) against things other than itself."""
import os

import numpy as np
import pytest

from oracle import tproduct as tp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _parse_slices(text, rows, cols):
    out = np.zeros((rows, cols, len(text.split("|"))))
    for k, sl in enumerate(text.split("|")):
        for r, row in enumerate(sl.split(";")):
            out[r, :, k] = [float(v) for v in row.split()]
    return out


def load_hand_cases():
    cases = []
    cur = None
    for line in open(os.path.join(GOLDEN, "tprod_hand.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tag, rest = line.split(None, 1)
        if tag == "case":
            name, n1, n2, m, p = rest.split()
            cur = dict(name=name, n1=int(n1), n2=int(n2), m=int(m), p=int(p))
            cases.append(cur)
        elif tag == "A":
            cur["A"] = _parse_slices(rest, cur["n1"], cur["n2"])
        elif tag == "B":
            cur["B"] = _parse_slices(rest, cur["n2"], cur["m"])
        elif tag == "C":
            cur["C"] = _parse_slices(rest, cur["n1"], cur["m"])
    return cases


@pytest.mark.parametrize("case", load_hand_cases(), ids=lambda c: c["name"])
def test_hand_computed(case):
    """Definition 2.1 worked by hand (tests/golden/tprod_hand.txt)."""
    for f in (tp.tprod_bcirc, tp.tprod_blockrow, tp.tprod):
        np.testing.assert_allclose(f(case["A"], case["B"]), case["C"], rtol=0, atol=1e-15)


def fft_tprod(A, B):
    """T-product through the block diagonalisation of Eq. (5), with numpy's FFT and all p slices."""
    Ah = np.fft.fft(A, axis=2)
    Bh = np.fft.fft(B, axis=2)
    return np.real(np.fft.ifft(np.einsum("ilk,ljk->ijk", Ah, Bh), axis=2))


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 7, 8, 16])
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 4, 2), (6, 5, 7)])
def test_tprod_matches_fft_route(p, shape):
    rng = np.random.default_rng(100 + p)
    n1, n2, m = shape
    A = rng.standard_normal((n1, n2, p))
    B = rng.standard_normal((n2, m, p))
    ref = fft_tprod(A, B)
    for f in (tp.tprod_bcirc, tp.tprod_blockrow):
        np.testing.assert_allclose(f(A, B), ref, rtol=0, atol=1e-12)


def test_blockrow_path_used_for_large():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 40, 40))   # bcirc would hold 2.56M entries * ... above the limit
    B = rng.standard_normal((40, 3, 40))
    np.testing.assert_allclose(tp.tprod(A, B), fft_tprod(A, B), rtol=0, atol=1e-10)


@pytest.mark.parametrize("p", [1, 2, 5, 8])
def test_p1_is_matrix_product_and_identity(p):
    rng = np.random.default_rng(p)
    A = rng.standard_normal((4, 3, 1))
    B = rng.standard_normal((3, 2, 1))
    np.testing.assert_allclose(tp.tprod(A, B)[:, :, 0], A[:, :, 0] @ B[:, :, 0], atol=1e-14)
    X = rng.standard_normal((5, 2, p))
    np.testing.assert_allclose(tp.tprod(tp.identity(5, p), X), X, atol=1e-15)
    np.testing.assert_allclose(tp.tprod(X, tp.identity(2, p)), X, atol=1e-15)


@pytest.mark.parametrize("p", [2, 3, 6])
def test_associativity_and_transpose_rule(p):
    """Definition 2.2(5) and 2.2(6)."""
    rng = np.random.default_rng(7 + p)
    A = rng.standard_normal((3, 4, p))
    B = rng.standard_normal((4, 5, p))
    C = rng.standard_normal((5, 2, p))
    np.testing.assert_allclose(tp.tprod(tp.tprod(A, B), C), tp.tprod(A, tp.tprod(B, C)), atol=1e-12)
    np.testing.assert_allclose(tp.ttranspose(tp.tprod(A, B)),
                               tp.tprod(tp.ttranspose(B), tp.ttranspose(A)), atol=1e-12)
    np.testing.assert_array_equal(tp.ttranspose(tp.ttranspose(A)), A)


def test_transpose_matches_bcirc_transpose():
    """bcirc(A^T) = bcirc(A)^T: the slice reversal of Definition 2.2(4) is the one that makes this hold."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((3, 4, 5))
    np.testing.assert_array_equal(tp.bcirc(tp.ttranspose(A)), tp.bcirc(A).T)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 8])
def test_dft3_matches_numpy_fft(p):
    rng = np.random.default_rng(p)
    A = rng.standard_normal((3, 2, p))
    np.testing.assert_allclose(tp.dft3(A), np.fft.fft(A, axis=2), atol=1e-13)
    np.testing.assert_allclose(tp.idft3(tp.dft3(A)), A, atol=1e-14)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_block_diagonalisation(p):
    """Eq. (5) with the unitary DFT matrix: (F x I) bcirc(A) (F^* x I) = Diag(A-hat)."""
    rng = np.random.default_rng(20 + p)
    n1, n2 = 3, 2
    A = rng.standard_normal((n1, n2, p))
    F = np.fft.fft(np.eye(p)) / np.sqrt(p)
    D = np.kron(F, np.eye(n1)) @ tp.bcirc(A) @ np.kron(F.conj().T, np.eye(n2))
    Ah = np.fft.fft(A, axis=2)
    expect = np.zeros((n1 * p, n2 * p), dtype=complex)
    for k in range(p):
        expect[k * n1:(k + 1) * n1, k * n2:(k + 1) * n2] = Ah[:, :, k]
    np.testing.assert_allclose(D, expect, atol=1e-12)


def test_tentry_matches_full_product():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((6, 4, 5))
    B = rng.standard_normal((4, 3, 5))
    C = fft_tprod(A, B)
    for (i, j, k) in [(0, 0, 0), (5, 2, 4), (3, 1, 2)]:
        assert abs(tp.tentry(A, B, i, j, k) - C[i, j, k]) < 1e-12


def test_inner_norm_tdiamond():
    rng = np.random.default_rng(9)
    As = [rng.standard_normal((3, 2, 4)) for _ in range(3)]
    G = tp.tdiamond(As, As)
    flat = np.stack([a.ravel() for a in As])
    np.testing.assert_allclose(G, flat @ flat.T, atol=1e-13)
    assert abs(tp.norm(As[0]) - np.linalg.norm(As[0].ravel())) < 1e-14


def test_tube_inverse():
    z = np.array([3.0, 1.0, -0.5, 0.25]).reshape(1, 1, 4)
    np.testing.assert_allclose(tp.tprod(z, tp.tube_inverse(z)), tp.tube_e(4), atol=1e-14)
    with pytest.raises(ZeroDivisionError):
        tp.tube_inverse(np.array([1.0, -1.0]).reshape(1, 1, 2))   # Fourier coefficient 0 at k = 0


def test_planted_mistake_is_caught(monkeypatch):
    """A wrong circulant direction in bcirc must fail the FFT pin (the pin can see such a mistake)."""
    def bad_bcirc(A):
        n1, n2, p = A.shape
        M = np.zeros((n1 * p, n2 * p))
        for r in range(p):
            for c in range(p):
                M[r * n1:(r + 1) * n1, c * n2:(c + 1) * n2] = A[:, :, (c - r) % p]
        return M
    monkeypatch.setattr(tp, "bcirc", bad_bcirc)
    rng = np.random.default_rng(1)
    A = rng.standard_normal((3, 3, 4))
    B = rng.standard_normal((3, 2, 4))
    assert np.abs(tp.tprod_bcirc(A, B) - fft_tprod(A, B)).max() > 1e-3
