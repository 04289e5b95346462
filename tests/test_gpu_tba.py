"""GPU parity of Tubal Block Arnoldi / TBAS(m), t-Bartels-Stewart and the sparse operator against the
oracle (Algorithms 5-8), through the C ABI.

Tolerances: residual histories |r_gpu - r_oracle| <= 1e-10 ||C|| per cycle (the same rule as the
tGMRES histories); solutions to 1e-9 relative; small direct solves (t-Bartels-Stewart) to 1e-10
relative to max |X| (the systems here have condition numbers below 1e2).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import krylov as kr, tproduct as tp, tubal as tb, schur as sc
from paper_2405_09233_gb300 import inputs
from tests.gpu_helpers import to_dev, from_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_09233_gb300 import Context
    c = Context(0)
    yield c
    c.workspace_check()          # no kernel wrote past the end of a workspace buffer
    c.close()


def csr_arrays(prob):
    """Concatenate the p CSR slices of a SparseProblem into the C-ABI layout."""
    n, p = prob.n, prob.p
    rowptr, cols, vals, base = [], [], [], 0
    for sl in prob.slices:
        rowptr.append(sl.rowptr.astype(np.int64) + base)
        cols.append(sl.col)
        vals.append(sl.val)
        base += sl.col.size
    return np.concatenate(rowptr).astype(np.int32), np.concatenate(cols), np.concatenate(vals)


def scipy_slices(prob):
    return [sp.csr_matrix((sl.val, sl.col, sl.rowptr), shape=(prob.n, prob.n)) for sl in prob.slices]


@pytest.mark.parametrize("dims", [(6, 3, 1), (8, 5, 2), (12, 4, 3), (20, 6, 4), (33, 7, 5), (16, 16, 8), (50, 2, 7),
                                  (8, 64, 2), (64, 64, 4), (128, 96, 4)],
                         ids=lambda d: "n%d_s%d_p%d" % d)
def test_t_bartels_stewart_matches_oracle(ctx, dims):
    """Up to mid sizes: (8, 64, 2) is a slice whose complex Schur iteration once stalled on its last 2 x 2
    window (fused multiply-add rounding kept the subdiagonal just above the deflation test)."""
    n, s, p = dims
    pr = inputs.dense_problem(n, s, p, seed=80 + n)
    C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
    X = from_dev(ctx.t_bartels_stewart(to_dev(pr.A), to_dev(pr.B), to_dev(C)))
    ref = sc.t_bartels_stewart(pr.A, pr.B, C)
    np.testing.assert_allclose(X, ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    np.testing.assert_allclose(X, pr.Xstar, rtol=0, atol=1e-10 * np.abs(pr.Xstar).max())


def test_t_bartels_stewart_singular_reported(ctx):
    """A = B: A_k and B_k share every eigenvalue, Theorem 2.1's condition fails."""
    n, p = 5, 3
    A = inputs.random_tensor((n, n, p), seed=3)
    C = inputs.random_tensor((n, n, p), seed=4)
    import torch
    X = torch.empty((p, n, n), dtype=torch.float64, device="cuda")
    from paper_2405_09233_gb300 import binding
    st = binding.lib().ts_t_bartels_stewart(ctx._h, to_dev(A).data_ptr(), n, to_dev(A).data_ptr(), n, p,
                                            to_dev(C).data_ptr(), X.data_ptr(), None)
    assert st == binding.TS_SINGULAR


@pytest.mark.parametrize("case", [(40, 4, 4, 4, 1), (30, 5, 5, 4, 2), (60, 3, 2, 6, 3), (64, 8, 8, 3, 4),
                                  (24, 24, 4, 3, 0), (256, 64, 4, 3, 6)], ids=lambda c: "n%d_s%d_p%d_m%d" % c[:4])
def test_tbas_dense_matches_oracle(ctx, case):
    import torch
    n, s, p, m, seed = case
    pr = inputs.dense_problem(n, s, p, seed=seed)
    C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
    ref = tb.tbas(pr.A, pr.B, C, m=m, tol=1e-10)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Xd = torch.zeros((p, s, n), dtype=torch.float64, device="cuda")
    res = ctx.tba_solve(op, to_dev(C), Xd, restart=m, tol=1e-10)
    X = from_dev(Xd)
    assert res.status == 0 and ref.status == "ok", (res, ref.status)
    assert len(res.true_history) == len(ref.true_res)
    np.testing.assert_allclose(res.true_history, ref.true_res, rtol=0, atol=1e-10 * ref.normC)
    np.testing.assert_allclose(res.history, ref.history, rtol=0, atol=1e-10 * ref.normC)
    np.testing.assert_allclose(X, ref.X, rtol=0, atol=1e-9 * np.abs(ref.X).max())
    assert tp.norm(C - kr.sylv_apply(pr.A, pr.B, X)) <= 1e-10 * tp.norm(C)
    op.close()


@pytest.mark.parametrize("shape", [(6, 3, 3), (12, 4, 4), (10, 8, 8), (20, 64, 4)], ids=lambda d: "grid%d_s%d_p%d" % d)
def test_sparse_operator_apply_and_tbas(ctx, shape):
    import torch
    grid, s, p = shape
    prob = inputs.sparse_problem(grid=grid, s=s, p=p, seed=5)
    slices = scipy_slices(prob)
    applyA = lambda Z: tb.tprod_sparse(slices, Z)  # noqa: E731
    rowptr, col, val = csr_arrays(prob)
    op = ctx.op_create_csr(prob.n, p, rowptr, col, val, to_dev(prob.B))
    X = inputs.random_tensor((prob.n, s, p), seed=9)
    Y = from_dev(ctx.sylv_apply(op, to_dev(X)))
    ref = applyA(X) - tp.tprod(X, prob.B)
    assert np.abs(Y - ref).max() <= 1e-12 * np.abs(ref).max()
    C = applyA(prob.Xstar) - tp.tprod(prob.Xstar, prob.B)
    r_ref = tb.tbas(None, prob.B, C, m=5, tol=1e-10, applyA=applyA)
    Xd = torch.zeros((p, s, prob.n), dtype=torch.float64, device="cuda")
    res = ctx.tba_solve(op, to_dev(C), Xd, restart=5, tol=1e-10)
    assert res.status == 0 and r_ref.status == "ok"
    np.testing.assert_allclose(res.true_history, r_ref.true_res, rtol=0, atol=1e-10 * r_ref.normC)
    np.testing.assert_allclose(from_dev(Xd), r_ref.X, rtol=0, atol=1e-9 * np.abs(r_ref.X).max())
    # the same sparse operator through restarted tGMRES
    g_ref = kr.tgmres(None, None, C, m=10, tol=1e-10, apply=lambda Z: applyA(Z) - tp.tprod(Z, prob.B))
    Xg = torch.zeros_like(Xd)
    g = ctx.tgmres_solve(op, to_dev(C), Xg, restart=10, tol=1e-10)
    assert g.status == 0 and len(g.history) == len(g_ref.history)
    np.testing.assert_allclose(g.history, g_ref.history, rtol=0, atol=1e-10 * g_ref.normC)
    op.close()


@pytest.mark.parametrize("s", [32, 4])
def test_tbas_sparse_full_size_lap128(ctx, s):
    """The sparse workload at full size: 5-point Laplacian on 128 x 128 plus 7 random slices, p = 8,
    block width s = 32 (and the s = 4 variant).  Sampled entries of M(X) against the oracle's
    single-entry definition, then TBAS(10) to a true relative residual of 1e-10."""
    import torch
    prob = inputs.sparse_problem(grid=128, s=s, p=8, seed=1)
    slices = scipy_slices(prob)
    rowptr, col, val = csr_arrays(prob)
    op = ctx.op_create_csr(prob.n, 8, rowptr, col, val, to_dev(prob.B))
    Xs = to_dev(prob.Xstar)
    Cd = ctx.sylv_apply(op, Xs)
    Y = from_dev(Cd)
    rng = np.random.default_rng(3)
    n, p = prob.n, 8
    for _ in range(30):
        i, j, k = int(rng.integers(n)), int(rng.integers(s)), int(rng.integers(p))
        ax = sum(slices[(k - c) % p].getrow(i).dot(prob.Xstar[:, j, c])[0] for c in range(p))
        xb = sum(prob.Xstar[i, :, (k - c) % p] @ prob.B[:, j, c] for c in range(p))
        assert abs(Y[i, j, k] - (ax - xb)) <= 1e-12 * (abs(ax) + abs(xb) + 1.0)
    Xd = torch.zeros_like(Cd)
    res = ctx.tba_solve(op, Cd, Xd, restart=10, tol=1e-10)
    assert res.status == 0, res
    R = Cd - ctx.sylv_apply(op, Xd)
    assert float(torch.linalg.norm(R) / torch.linalg.norm(Cd)) <= 1e-10
    assert float(torch.max(torch.abs(Xd - Xs))) < 1e-8
    op.close()


@pytest.mark.parametrize("case", [(40, 4, 4, 4, 1), (60, 3, 2, 6, 3), (64, 8, 8, 3, 4), (24, 24, 4, 3, 0)],
                         ids=lambda c: "n%d_s%d_p%d_m%d" % c[:4])
def test_tbas_mixed_fp32_dense(ctx, case):
    """Mixed-precision TBAS (FP32 block Krylov cycles, FP64 residuals and solution) reaches a true
    relative residual of 1e-10 and the oracle's FP64 TBAS solution."""
    import torch
    n, s, p, m, seed = case
    pr = inputs.dense_problem(n, s, p, seed=seed)
    C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
    ref = tb.tbas(pr.A, pr.B, C, m=m, tol=1e-10)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Xd = torch.zeros((p, s, n), dtype=torch.float64, device="cuda")
    res = ctx.tba_solve(op, to_dev(C), Xd, restart=m, tol=1e-10, precision="mixed_fp32")
    X = from_dev(Xd)
    assert res.status == 0, res
    assert tp.norm(C - kr.sylv_apply(pr.A, pr.B, X)) <= 1e-10 * tp.norm(C)
    np.testing.assert_allclose(X, ref.X, rtol=0, atol=1e-8 * np.abs(ref.X).max())
    assert res.info.applies_low > 0 and res.info.outer == res.info.cycles
    op.close()


@pytest.mark.parametrize("s", [32, 4])
def test_tbas_mixed_fp32_sparse_lap128(ctx, s):
    """The sparse workload at full size with mixed-precision TBAS(10): true relative residual
    1e-10 (FP64 operator) and the manufactured solution."""
    import torch
    prob = inputs.sparse_problem(grid=128, s=s, p=8, seed=1)
    rowptr, col, val = csr_arrays(prob)
    op = ctx.op_create_csr(prob.n, 8, rowptr, col, val, to_dev(prob.B))
    Xs = to_dev(prob.Xstar)
    Cd = ctx.sylv_apply(op, Xs)
    Xd = torch.zeros_like(Cd)
    res = ctx.tba_solve(op, Cd, Xd, restart=10, tol=1e-10, precision="mixed_fp32")
    assert res.status == 0, res
    R = Cd - ctx.sylv_apply(op, Xd)
    assert float(torch.linalg.norm(R) / torch.linalg.norm(Cd)) <= 1e-10
    assert float(torch.max(torch.abs(Xd - Xs))) < 1e-8
    op.close()



def deficient_rhs(n, s, p, kind, seed):
    """A random right-hand side whose lateral slice 1 repeats slice 0 ("equal") or is zero ("zero")."""
    C = inputs.random_tensor((n, s, p), seed=seed)
    C[:, 1, :] = C[:, 0, :] if kind == "equal" else 0.0
    return C


@pytest.mark.parametrize("kind", ["equal", "zero"])
@pytest.mark.parametrize("case", [(20, 3, 4, 3), (40, 4, 5, 4), (33, 6, 8, 3)], ids=lambda c: "n%d_s%d_p%d_m%d" % c)
def test_tbas_rank_deficient_start_dense(ctx, case, kind):
    """R0 = C with a repeated or zero lateral slice: Tubal-QR's first block is rank deficient in every
    Fourier slice, the GPU takes Algorithm 6 with the Normalize tie-break there (not CholeskyQR2),
    and TBAS(m) follows the oracle's residual histories and solution."""
    import torch
    n, s, p, m = case
    pr = inputs.dense_problem(n, s, p, seed=5)
    C = deficient_rhs(n, s, p, kind, seed=6)
    ref = tb.tbas(pr.A, pr.B, C, m=m, tol=1e-10)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Xd = torch.zeros((p, s, n), dtype=torch.float64, device="cuda")
    res = ctx.tba_solve(op, to_dev(C), Xd, restart=m, tol=1e-10)
    X = from_dev(Xd)
    assert res.status == 0 and ref.status == "ok", (res, ref.status)
    assert len(res.true_history) == len(ref.true_res)
    np.testing.assert_allclose(res.true_history, ref.true_res, rtol=0, atol=1e-10 * ref.normC)
    np.testing.assert_allclose(res.history, ref.history, rtol=0, atol=1e-10 * ref.normC)
    np.testing.assert_allclose(X, ref.X, rtol=0, atol=1e-9 * np.abs(ref.X).max())
    op.close()


@pytest.mark.parametrize("kind", ["equal", "zero"])
def test_tbas_rank_deficient_start_sparse(ctx, kind):
    import torch
    grid, s, p, m = 6, 3, 3, 5
    prob = inputs.sparse_problem(grid=grid, s=s, p=p, seed=5)
    slices = scipy_slices(prob)
    applyA = lambda Z: tb.tprod_sparse(slices, Z)  # noqa: E731
    rowptr, col, val = csr_arrays(prob)
    op = ctx.op_create_csr(prob.n, p, rowptr, col, val, to_dev(prob.B))
    C = deficient_rhs(prob.n, s, p, kind, seed=8)
    ref = tb.tbas(None, prob.B, C, m=m, tol=1e-10, applyA=applyA)
    Xd = torch.zeros((p, s, prob.n), dtype=torch.float64, device="cuda")
    res = ctx.tba_solve(op, to_dev(C), Xd, restart=m, tol=1e-10)
    assert res.status == 0 and ref.status == "ok", (res, ref.status)
    assert len(res.true_history) == len(ref.true_res)
    np.testing.assert_allclose(res.true_history, ref.true_res, rtol=0, atol=1e-10 * ref.normC)
    np.testing.assert_allclose(res.history, ref.history, rtol=0, atol=1e-10 * ref.normC)
    np.testing.assert_allclose(from_dev(Xd), ref.X, rtol=0, atol=1e-9 * np.abs(ref.X).max())
    op.close()


def test_tbas_mixed_rank_deficient_start_converges(ctx):
    """The FP32 inner cycle of mixed-precision TBAS takes the same fallback and still reaches 1e-10."""
    import torch
    n, s, p, m = 40, 4, 5, 4
    pr = inputs.dense_problem(n, s, p, seed=5)
    C = deficient_rhs(n, s, p, "zero", seed=6)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Xd = torch.zeros((p, s, n), dtype=torch.float64, device="cuda")
    res = ctx.tba_solve(op, to_dev(C), Xd, restart=m, tol=1e-10, precision="mixed_fp32")
    assert res.status == 0, res
    assert tp.norm(C - kr.sylv_apply(pr.A, pr.B, from_dev(Xd))) <= 1e-10 * tp.norm(C)
    op.close()
