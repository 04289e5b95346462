"""Pins for the oracle's Sylvester operator, tArnoldi, tFOM and tGMRES (§3)."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

from oracle import tproduct as tp, krylov as kr
from paper_2405_09233_gb300 import inputs


def kron_matrix(A, B):
    """Matrix of M acting on vec(unfold(X)), derived from Definition 2.1 by hand.

    unfold(A*X) = bcirc(A) unfold(X) gives I_s (x) bcirc(A).  Block k of
    unfold(X*B) is sum_c X^((k-c) mod p) B^(c) = sum_c (S_c unfold(X)) B^(c), with
    S_c the block shift taking block k-c to block k, so vec(unfold(X*B)) =
    sum_c (B^(c)^T (x) S_c) vec(unfold(X)).
    """
    n, _, p = A.shape
    s = B.shape[0]
    K = np.kron(np.eye(s), tp.bcirc(A))
    for c in range(p):
        S = np.zeros((n * p, n * p))
        for k in range(p):
            r = (k - c) % p
            S[k * n:(k + 1) * n, r * n:(r + 1) * n] = np.eye(n)
        K -= np.kron(B[:, :, c].T, S)
    return K


def vec(X):
    return tp.unfold(X).ravel(order="F")


def unvec(u, n, s, p):
    return tp.fold(u.reshape((n * p, s), order="F"), p)


def fourier_solve(A, B, C):
    """Theorem 2.1's route: per Fourier slice, solve A_k X_k - X_k B_k = C_k by a Kronecker system."""
    n, s, p = C.shape
    Ah, Bh, Ch = (np.fft.fft(T, axis=2) for T in (A, B, C))
    Xh = np.zeros((n, s, p), dtype=complex)
    for k in range(p):
        Kk = np.kron(np.eye(s), Ah[:, :, k]) - np.kron(Bh[:, :, k].T, np.eye(n))
        Xh[:, :, k] = np.linalg.solve(Kk, Ch[:, :, k].ravel(order="F")).reshape((n, s), order="F")
    return np.real(np.fft.ifft(Xh, axis=2))


@pytest.mark.parametrize("dims", [(4, 3, 1), (5, 2, 2), (4, 3, 3), (3, 4, 4), (2, 2, 5)])
def test_apply_matches_kronecker_matrix(dims):
    n, s, p = dims
    pr = inputs.dense_problem(n, s, p, seed=40 + p)
    X = inputs.random_tensor((n, s, p), seed=1)
    K = kron_matrix(pr.A, pr.B)
    np.testing.assert_allclose(vec(kr.sylv_apply(pr.A, pr.B, X)), K @ vec(X), atol=1e-12)


def test_apply_matches_fft_route():
    pr = inputs.dense_problem(7, 5, 6, seed=3)
    X = inputs.random_tensor((7, 5, 6), seed=2)
    Ah, Bh, Xh = (np.fft.fft(T, axis=2) for T in (pr.A, pr.B, X))
    Yh = np.einsum("ilk,ljk->ijk", Ah, Xh) - np.einsum("ilk,ljk->ijk", Xh, Bh)
    np.testing.assert_allclose(kr.sylv_apply(pr.A, pr.B, X), np.real(np.fft.ifft(Yh, axis=2)), atol=1e-12)


def test_workload_n24_kronecker_solve_recovers_xstar():
    """The 24 x 24 x 4 dense workload: dense solve of size 2304 and the Fourier route both give X*."""
    pr = inputs.dense_problem(24, 24, 4, seed=0)
    C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
    K = kron_matrix(pr.A, pr.B)
    X = unvec(np.linalg.solve(K, vec(C)), 24, 24, 4)
    assert np.abs(X - pr.Xstar).max() < 1e-12
    assert np.abs(fourier_solve(pr.A, pr.B, C) - pr.Xstar).max() < 1e-12


@pytest.mark.parametrize("m", [3, 5, 20])
def test_tgmres_history_matches_scipy_gmres(m):
    """tGMRES(m) is restarted GMRES on vec(X) with the Euclidean inner product (Definition 2.3)."""
    n, s, p = 8, 6, 3
    pr = inputs.dense_problem(n, s, p, seed=11)
    C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
    K = kron_matrix(pr.A, pr.B)
    hist = []
    sla.gmres(K, vec(C), restart=m, rtol=1e-10, atol=0.0, maxiter=200,
              callback=lambda r: hist.append(r), callback_type="pr_norm")
    res = kr.tgmres(pr.A, pr.B, C, m=m, tol=1e-10)
    assert res.status == "ok" and res.relres <= 1e-10
    h = np.array(res.history) / res.normC
    assert len(h) == len(hist)
    np.testing.assert_allclose(h, hist, rtol=0, atol=1e-12)


def test_workload_n24_tgmres_tfom_converge():
    pr = inputs.dense_problem(24, 24, 4, seed=0)
    C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
    g = kr.tgmres(pr.A, pr.B, C, m=20, tol=1e-10)
    f = kr.tfom(pr.A, pr.B, C, m=20, tol=1e-10)
    for r in (g, f):
        assert r.status == "ok" and r.relres <= 1e-10
        assert np.abs(r.X - pr.Xstar).max() < 1e-8
    # GMRES residual estimates never increase within a cycle.
    assert all(b <= a * (1 + 1e-12) for a, b in zip(g.history, g.history[1:]))


def test_arnoldi_relations():
    """Propositions 3.1 and 3.2.

    Modified Gram-Schmidt loses orthogonality in proportion to u / (relative
    residual), so 1e-12 orthonormality is checked on a basis whose residual is
    still large (m = 6 here); the Arnoldi relation holds to rounding at any m.
    """
    pr = inputs.dense_problem(6, 5, 4, seed=5)
    apply = lambda X: kr.sylv_apply(pr.A, pr.B, X)  # noqa: E731
    V0 = inputs.random_tensor((6, 5, 4), seed=6)
    m = 6
    Vs, Ht, beta = kr.tarnoldi(apply, V0, m)
    assert len(Vs) == m + 1
    G = tp.tdiamond(Vs, Vs)
    assert np.abs(G - np.eye(m + 1)).max() < 1e-12                     # V^T <> V = I
    Ws = [apply(V) for V in Vs[:m]]
    for j in range(m):                                                # W_m = V_{m+1} (*) Htilde_m
        assert tp.norm(Ws[j] - kr.combine(Vs, Ht[:, j])) < 1e-12 * tp.norm(Ws[j])
    np.testing.assert_allclose(tp.tdiamond(Vs[:m], Ws), Ht[:m, :], atol=1e-12)   # V_m^T <> W_m = H_m
    y = np.random.default_rng(0).standard_normal(m)
    assert abs(tp.norm(kr.combine(Vs[:m], y)) - np.linalg.norm(y)) < 1e-12     # Proposition 3.1


@pytest.mark.parametrize("method", ["fom", "gmres"])
def test_estimate_equals_true_residual(method):
    """Propositions 3.3 (tFOM) and 3.4 (tGMRES): the cheap estimate is the true residual norm."""
    pr = inputs.dense_problem(7, 4, 3, seed=8)
    C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
    for m in range(1, 9):
        r = kr.restarted_solve(method, pr.A, pr.B, C, m=m, tol=1e-300, max_restarts=1)
        assert abs(r.history[-1] - r.true_res[-1]) <= 1e-11 * r.normC


def test_fom_gmres_relation():
    """||r^F_j|| = ||r^G_j|| / sqrt(1 - (||r^G_j|| / ||r^G_{j-1}||)^2) within one cycle (Brown 1991)."""
    pr = inputs.dense_problem(9, 4, 2, seed=9)
    C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
    g = kr.tgmres(pr.A, pr.B, C, m=10, tol=1e-300, max_restarts=1).history
    f = kr.tfom(pr.A, pr.B, C, m=10, tol=1e-300, max_restarts=1).history
    gprev = [np.linalg.norm(C)] + g[:-1]
    for j in range(len(g)):
        pred = g[j] / np.sqrt(1.0 - (g[j] / gprev[j]) ** 2)
        assert abs(f[j] - pred) <= 1e-8 * pred


def test_breakdown_gives_exact_solution():
    """C in a 1-dimensional invariant subspace of M: Arnoldi breaks down at j = 1, tGMRES is exact."""
    n, s, p = 4, 3, 2
    A = np.zeros((n, n, p)); A[:, :, 0] = 3.0 * np.eye(n)
    B = np.zeros((s, s, p)); B[:, :, 0] = -np.eye(s)
    C = inputs.random_tensor((n, s, p), seed=1)        # M = 4 I, so M(C) is parallel to C
    r = kr.tgmres(A, B, C, m=5, tol=1e-10)
    assert r.iters == 1 and r.status == "ok"
    np.testing.assert_allclose(r.X, C / 4.0, atol=1e-15)


def test_planted_sign_mistake_is_caught(monkeypatch):
    """A '+' in the operator must fail the Kronecker pin."""
    pr = inputs.dense_problem(4, 3, 3, seed=2)
    X = inputs.random_tensor((4, 3, 3), seed=3)
    K = kron_matrix(pr.A, pr.B)
    monkeypatch.setattr(kr, "sylv_apply", lambda A, B, X: tp.tprod(A, X) + tp.tprod(X, B))
    assert np.abs(vec(kr.sylv_apply(pr.A, pr.B, X)) - K @ vec(X)).max() > 1e-3
