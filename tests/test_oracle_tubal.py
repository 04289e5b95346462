"""Pins for Normalize, Tubal-QR, TBA, TBAS (§5) and t-Schur / t-Bartels-Stewart (§4)."""
import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp

from oracle import tproduct as tp, krylov as kr, tubal as tb, schur as sc
from paper_2405_09233_gb300 import inputs
from tests.test_oracle_krylov import fourier_solve


@pytest.mark.parametrize("p", [1, 2, 3, 4, 8])
def test_normalize(p):
    """v = u * a and u^T * u = e (the Normalization1 property the paper states)."""
    v = inputs.random_tensor((7, 1, p), seed=p)
    u, a = tb.normalize(v)
    np.testing.assert_allclose(tp.tprod(u, a), v, atol=1e-14)
    np.testing.assert_allclose(tp.tprod(tp.ttranspose(u), u), tp.tube_e(p), atol=1e-14)
    if p == 1:   # reduces to v / ||v||
        np.testing.assert_allclose(u[:, 0, 0], v[:, 0, 0] / np.linalg.norm(v), atol=1e-15)


def test_normalize_rank_deficient_tube():
    """A lateral slice whose Fourier coefficient vanishes at k = 0 takes the e_1 tie-break there."""
    v = np.zeros((3, 1, 2))
    v[:, 0, 0] = [1.0, 2.0, 0.5]
    v[:, 0, 1] = -v[:, 0, 0]             # v-hat_0 = 0
    u, a = tb.normalize(v)
    np.testing.assert_allclose(tp.tprod(u, a), v, atol=1e-14)
    np.testing.assert_allclose(tp.tprod(tp.ttranspose(u), u), tp.tube_e(2), atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 5])
def test_tubal_qr(p):
    """Theorem 5.1 / Algorithm 6: A = Q * R, Q^T * Q = I, R upper triangular in tubes."""
    Amat = inputs.random_tensor((9, 4, p), seed=10 + p)
    Q, R = tb.tubal_qr(Amat)
    np.testing.assert_allclose(tp.tprod(Q, R), Amat, atol=1e-13)
    np.testing.assert_allclose(tp.tprod(tp.ttranspose(Q), Q), tp.identity(4, p), atol=1e-13)
    for i in range(4):
        for j in range(i):
            assert np.abs(R[i, j, :]).max() == 0.0
    if p == 1:   # thin QR with a positive diagonal
        q, r = np.linalg.qr(Amat[:, :, 0])
        sgn = np.sign(np.diag(r))
        np.testing.assert_allclose(Q[:, :, 0], q * sgn, atol=1e-13)
        np.testing.assert_allclose(R[:, :, 0], sgn[:, None] * r, atol=1e-13)


def block_arnoldi_matrix(A, V, m):
    """Textbook block Arnoldi (thin QR with a positive diagonal) for p = 1."""
    Q0, H0 = np.linalg.qr(V)
    d = np.sign(np.diag(H0)); Q0, H0 = Q0 * d, d[:, None] * H0
    Qs, s = [Q0], V.shape[1]
    Hbig = np.zeros(((m + 1) * s, m * s))
    for j in range(m):
        W = A @ Qs[j]
        for i in range(j + 1):
            h = Qs[i].T @ W
            Hbig[i * s:(i + 1) * s, j * s:(j + 1) * s] = h
            W = W - Qs[i] @ h
        q, r = np.linalg.qr(W)
        d = np.sign(np.diag(r)); q, r = q * d, d[:, None] * r
        Hbig[(j + 1) * s:(j + 2) * s, j * s:(j + 1) * s] = r
        Qs.append(q)
    return Qs, Hbig


def test_tba_p1_is_block_arnoldi():
    """With p = 1 Algorithm 7 is the block Arnoldi process (the remark after Proposition 5.1)."""
    n, s, m = 12, 3, 3
    A = inputs.random_tensor((n, n, 1), seed=1)
    V = inputs.random_tensor((n, s, 1), seed=2)
    arn = tb.tba(lambda X: tp.tprod(A, X), V, m)
    Qs, Hbig = block_arnoldi_matrix(A[:, :, 0], V[:, :, 0], m)
    for j in range(m + 1):
        np.testing.assert_allclose(arn.V[j][:, :, 0], Qs[j], atol=1e-12)
    np.testing.assert_allclose(arn.Hm()[:, :, 0], Hbig[:m * s, :], atol=1e-12)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_tba_relations(p):
    """Proposition 5.1: A*V_m = V_m*H_m + V_{m+1}*(H_{m+1,m}*E_m), V_m^T*A*V_m = H_m, V_m^T*V_m = I."""
    n, s, m = 20, 3, 3
    A = inputs.random_tensor((n, n, p), seed=30 + p)
    V = inputs.random_tensor((n, s, p), seed=31 + p)
    arn = tb.tba(lambda X: tp.tprod(A, X), V, m)
    Vm, Hm = arn.Vm(), arn.Hm()
    E = np.zeros((s, m * s, p)); E[:, (m - 1) * s:, :] = tp.identity(s, p)
    lhs = tp.tprod(A, Vm)
    rhs = tp.tprod(Vm, Hm) + tp.tprod(arn.V[m], tp.tprod(arn.H[(m, m - 1)], E))
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)
    np.testing.assert_allclose(tp.tprod(tp.ttranspose(Vm), lhs), Hm, atol=1e-12)
    np.testing.assert_allclose(tp.tprod(tp.ttranspose(Vm), Vm), tp.identity(m * s, p), atol=1e-12)
    np.testing.assert_allclose(tp.tprod(arn.V[0], arn.H0), V, atol=1e-13)


def test_tbas_converges_and_estimate_is_true_residual():
    """Algorithm 8 on a small dense problem; Proposition 5.2 holds every cycle."""
    pr = inputs.dense_problem(40, 4, 4, seed=1)
    C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
    r = tb.tbas(pr.A, pr.B, C, m=4, tol=1e-10)
    assert r.status == "ok" and r.relres <= 1e-10
    assert np.abs(r.X - fourier_solve(pr.A, pr.B, C)).max() < 1e-9
    for est, true in zip(r.history, r.true_res[1:]):
        assert abs(est - true) <= 1e-12 * r.normC + 1e-6 * true


def test_tbas_sparse_matches_dense():
    """The sparse family's structure on a 6 x 6 grid: sparse and dense T-products agree, TBAS converges."""
    prob = inputs.sparse_problem(grid=6, s=3, p=3, seed=4)
    Ad = prob.dense_A()
    slices = [sp.csr_matrix((sl.val, sl.col, sl.rowptr), shape=(prob.n, prob.n)) for sl in prob.slices]
    X = prob.Xstar
    np.testing.assert_allclose(tb.tprod_sparse(slices, X), tp.tprod(Ad, X), atol=1e-13)
    C = kr.sylv_apply(Ad, prob.B, prob.Xstar)
    r = tb.tbas(None, prob.B, C, m=5, tol=1e-10, applyA=lambda Z: tb.tprod_sparse(slices, Z))
    assert r.status == "ok" and np.abs(r.X - prob.Xstar).max() < 1e-8


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_t_schur(p):
    """Theorem 4.1 / Algorithm 4 (complex reading): A = U*R*U^H, U^H*U = I, R upper triangular."""
    A = inputs.random_tensor((5, 5, p), seed=50 + p)
    U, R = sc.t_schur(A)
    np.testing.assert_allclose(tp.tprod(tp.tprod(U, R), tp.cttranspose(U)), A, atol=1e-12)
    np.testing.assert_allclose(tp.tprod(tp.cttranspose(U), U), tp.identity(5, p), atol=1e-12)
    for i in range(5):
        for j in range(i):
            assert np.abs(R[i, j, :]).max() < 1e-13


def test_t_bartels_stewart_p1_is_solve_sylvester():
    A = inputs.random_tensor((6, 6, 1), seed=1) + 4 * np.eye(6)[:, :, None]
    B = inputs.random_tensor((3, 3, 1), seed=2) - 4 * np.eye(3)[:, :, None]
    C = inputs.random_tensor((6, 3, 1), seed=3)
    X = sc.t_bartels_stewart(A, B, C)
    ref = scipy.linalg.solve_sylvester(A[:, :, 0], -B[:, :, 0], C[:, :, 0])
    np.testing.assert_allclose(X[:, :, 0], ref, atol=1e-13)


@pytest.mark.parametrize("dims", [(5, 3, 2), (4, 4, 3), (6, 2, 4), (3, 5, 5)])
def test_t_bartels_stewart_matches_fourier_solve(dims):
    n, s, p = dims
    pr = inputs.dense_problem(n, s, p, seed=60 + p)
    C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
    X, imag = sc.t_bartels_stewart(pr.A, pr.B, C, return_imag=True)
    assert imag < 1e-12
    np.testing.assert_allclose(X, pr.Xstar, atol=1e-12)
    np.testing.assert_allclose(X, fourier_solve(pr.A, pr.B, C), atol=1e-12)


def deficient_block(n, p, seed):
    """A random n x 4 x p block whose lateral slice 2 equals slice 0 and whose slice 3 is zero."""
    Amat = inputs.random_tensor((n, 4, p), seed=seed)
    Amat[:, 2, :] = Amat[:, 0, :]
    Amat[:, 3, :] = 0.0
    return Amat


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_tubal_qr_rank_deficient(p):
    """Theorem 5.1 for a rank-deficient block: Q * R = A and Q^T * Q = I still hold, the dependent
    and the zero column get an exactly zero diagonal tube in R, and the zero column an exactly zero
    column of R."""
    Amat = deficient_block(9, p, seed=20 + p)
    Q, R = tb.tubal_qr(Amat)
    np.testing.assert_allclose(tp.tprod(Q, R), Amat, atol=1e-13)
    np.testing.assert_allclose(tp.tprod(tp.ttranspose(Q), Q), tp.identity(4, p), atol=1e-13)
    assert np.all(R[2, 2, :] == 0.0) and np.all(R[3, 3, :] == 0.0)
    assert np.all(R[:, 3, :] == 0.0)
    for i in range(4):
        for j in range(i):
            assert np.abs(R[i, j, :]).max() == 0.0
    if p == 1:   # the independent columns: thin QR with a positive diagonal
        q, r = np.linalg.qr(Amat[:, :2, 0])
        sgn = np.sign(np.diag(r))
        np.testing.assert_allclose(Q[:, :2, 0], q * sgn, atol=1e-13)


def test_tubal_qr_deficient_column_does_not_follow_rounding_noise():
    """The dependent column's Q does not depend on the rounding noise its orthogonalisation leaves:
    a copy of slice 0 and a copy scaled by (1 + 2^-52) give the same Q to rounding."""
    Amat = deficient_block(11, 3, seed=7)
    Q1, R1 = tb.tubal_qr(Amat)
    A2 = Amat.copy()
    A2[:, 2, :] = Amat[:, 0, :] * (1.0 + 2.0 ** -52)
    Q2, R2 = tb.tubal_qr(A2)
    np.testing.assert_allclose(Q2, Q1, atol=1e-14)
    np.testing.assert_allclose(R2, R1, atol=1e-14)


def test_completion_vector_skips_spanned_unit_vectors():
    """When e_1 lies in the span of the previous columns the next qualifying e_i is taken."""
    P = np.zeros((5, 2), dtype=complex)
    P[0, 0] = 1.0                       # e_1 itself
    P[1, 1] = 1j                        # a phase of e_2
    z = tb.completion_vector(P)
    np.testing.assert_allclose(z, np.eye(5)[2], atol=1e-15)


@pytest.mark.parametrize("kind", ["equal", "zero"])
def test_tba_and_tbas_with_rank_deficient_start(kind):
    """Algorithm 7 from a rank-deficient R0 keeps Proposition 5.1's identities, and TBAS(m) (Algorithm 8)
    solves the equation: a right-hand side whose lateral slice 2 equals slice 1, or whose slice 2 is zero."""
    n, s, p, m = 20, 3, 4, 3
    pr = inputs.dense_problem(n, s, p, seed=5)
    C = inputs.random_tensor((n, s, p), seed=6)
    if kind == "equal":
        C[:, 1, :] = C[:, 0, :]
    else:
        C[:, 1, :] = 0.0
    arn = tb.tba(lambda X: tp.tprod(pr.A, X), C, m)
    Vm, Hm = arn.Vm(), arn.Hm()
    np.testing.assert_allclose(tp.tprod(tp.ttranspose(Vm), Vm), tp.identity(m * s, p), atol=1e-12)
    np.testing.assert_allclose(tp.tprod(tp.ttranspose(Vm), tp.tprod(pr.A, Vm)), Hm, atol=1e-12)
    np.testing.assert_allclose(tp.tprod(arn.V[0], arn.H0), C, atol=1e-13)
    r = tb.tbas(pr.A, pr.B, C, m=m, tol=1e-10)
    assert r.status == "ok" and r.relres <= 1e-10
    assert np.abs(r.X - fourier_solve(pr.A, pr.B, C)).max() < 1e-9
