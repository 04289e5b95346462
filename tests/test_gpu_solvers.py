"""GPU parity of restarted tGMRES / tFOM (FP64 and mixed precision) against the oracle, through the C ABI.

Tolerances.  Residual histories: |h_gpu(j) - h_oracle(j)| <= 1e-10 ||C|| at every inner step
(values near 1e-10 ||C|| cannot agree to 1e-10 relative to themselves).  Solutions: the true
relative residual ||C - M(X)|| / ||C|| <= 1e-10, computed by the oracle at small sizes and by the
library's FP64 operator (itself pinned by test_gpu_apply) at full size.
"""
import numpy as np
import pytest

from oracle import krylov as kr, tproduct as tp
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


def run(ctx, method, pr, m, tol=1e-10, max_restarts=200, X0=None, **kw):
    import torch
    C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Xd = to_dev(np.zeros_like(C) if X0 is None else X0)
    fn = ctx.tgmres_solve if method == "gmres" else ctx.tfom_solve
    res = fn(op, to_dev(C), Xd, restart=m, tol=tol, max_restarts=max_restarts, **kw)
    torch.cuda.synchronize()
    X = from_dev(Xd)
    op.close()
    return C, X, res


CASES = [  # (n, s, p, m, seed)
    (24, 24, 4, 20, 0),      # the 24 x 24 x 4 dense workload, tGMRES(20)
    (24, 24, 4, 5, 0),       # same, short restarts (several cycles)
    (37, 5, 7, 8, 3),        # ragged, odd p
    (16, 9, 1, 10, 4),       # p = 1 (matrix Sylvester equation)
    (70, 66, 16, 12, 5),     # two 64-tiles in both dimensions
    (40, 48, 16, 15, 6),     # 30720 unknowns: the one-launch step tail with 8 entries per thread
    (60, 64, 16, 12, 7),     # 61440 unknowns: 16 entries per thread
]


@pytest.mark.parametrize("method", ["gmres", "fom"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "n%d_s%d_p%d_m%d" % c[:4])
def test_fp64_history_parity(ctx, method, case):
    n, s, p, m, seed = case
    pr = inputs.dense_problem(n, s, p, seed=seed)
    C, X, res = run(ctx, method, pr, m)
    ref = kr.restarted_solve(method, pr.A, pr.B, C, m=m, tol=1e-10)
    assert res.status == 0 and ref.status == "ok"
    assert len(res.history) == len(ref.history), (len(res.history), len(ref.history))
    np.testing.assert_allclose(res.history, ref.history, rtol=0, atol=1e-10 * ref.normC)
    np.testing.assert_allclose(res.true_history, ref.true_res, rtol=0, atol=1e-10 * ref.normC)
    assert tp.norm(C - kr.sylv_apply(pr.A, pr.B, X)) <= 1e-10 * tp.norm(C)
    assert np.abs(X - ref.X).max() <= 1e-8 * np.abs(ref.X).max()
    assert res.info.iters == ref.iters and res.info.cycles == ref.cycles


@pytest.mark.parametrize("method", ["gmres", "fom"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "n%d_s%d_p%d_m%d" % c[:4])
def test_fp64_spectral_basis_history_parity(ctx, method, case):
    """The Krylov basis kept in the Fourier domain (scaled half spectrum, Parseval inner product): the
    same iterates as the real-space basis, so the oracle's residual histories, cycles and solution."""
    n, s, p, m, seed = case
    pr = inputs.dense_problem(n, s, p, seed=seed)
    C, X, res = run(ctx, method, pr, m, spectral=True)
    ref = kr.restarted_solve(method, pr.A, pr.B, C, m=m, tol=1e-10)
    assert res.status == 0 and ref.status == "ok"
    assert len(res.history) == len(ref.history), (len(res.history), len(ref.history))
    np.testing.assert_allclose(res.history, ref.history, rtol=0, atol=1e-10 * ref.normC)
    np.testing.assert_allclose(res.true_history, ref.true_res, rtol=0, atol=1e-10 * ref.normC)
    assert tp.norm(C - kr.sylv_apply(pr.A, pr.B, X)) <= 1e-10 * tp.norm(C)
    assert np.abs(X - ref.X).max() <= 1e-8 * np.abs(ref.X).max()
    assert res.info.iters == ref.iters and res.info.cycles == ref.cycles


def test_spectral_basis_rejected_where_unsupported(ctx):
    import torch
    from paper_2405_09233_gb300 import TstarError
    pr = inputs.dense_problem(8, 4, 3, seed=1)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    C = to_dev(inputs.random_tensor((8, 4, 3), seed=2))
    with pytest.raises(TstarError) as e:
        ctx.tgmres_solve(op, C, torch.zeros_like(C), restart=5, precision="mixed_fp32", spectral=True)
    assert e.value.status == -6                            # TS_ERR_UNSUPPORTED
    op.close()


@pytest.mark.parametrize("method", ["gmres", "fom"])
@pytest.mark.parametrize("case", [(24, 24, 4, 20, 0), (24, 24, 4, 5, 0), (37, 5, 7, 8, 3), (70, 66, 16, 4, 5)],
                         ids=lambda c: "n%d_s%d_p%d_m%d" % c[:4])
def test_execution_forms_agree_bitwise(ctx, monkeypatch, method, case):
    """A small problem's cycle launched ahead behind a device gate (<= 65536 unknowns) and a larger one's
    cycle replayed as a conditional CUDA graph (from the second cycle on) run the same kernels in the same
    order as the per-step host loop: identical histories, cycle counts and X, bit for bit."""
    n, s, p, m, seed = case
    pr = inputs.dense_problem(n, s, p, seed=seed)
    _, X1, r1 = run(ctx, method, pr, m)
    monkeypatch.setenv("TSTAR_NO_LAUNCH_AHEAD" if n * s * p <= 65536 else "TSTAR_NO_GRAPH_CYCLE", "1")
    _, X2, r2 = run(ctx, method, pr, m)
    assert r1.status == r2.status == 0
    assert r1.info.iters == r2.info.iters and r1.info.cycles == r2.info.cycles
    assert np.array_equal(np.asarray(r1.history), np.asarray(r2.history))
    assert np.array_equal(np.asarray(r1.true_history), np.asarray(r2.true_history))
    assert np.array_equal(X1, X2)
    if n * s * p > 65536:
        assert r1.info.cycles >= 2     # the graph form was exercised


def test_fp64_deterministic_and_resumable(ctx):
    """Fixed-order reductions: two runs are bitwise equal, and stopping after two cycles then
    resuming from the returned X (the restart state of Algorithm 3) reproduces the full run."""
    pr = inputs.dense_problem(24, 24, 4, seed=0)
    C, X1, r1 = run(ctx, "gmres", pr, 5)
    _, X2, r2 = run(ctx, "gmres", pr, 5)
    np.testing.assert_array_equal(X1, X2)
    np.testing.assert_array_equal(r1.history, r2.history)
    _, Xa, ra = run(ctx, "gmres", pr, 5, max_restarts=2)
    assert ra.status == 2 and ra.info.cycles == 2
    _, Xb, rb = run(ctx, "gmres", pr, 5, X0=Xa)
    assert rb.status == 0
    np.testing.assert_array_equal(Xb, X1)


@pytest.mark.parametrize("shape", [(24, 24, 4, 20), (65, 40, 8, 20), (200, 30, 16, 30)],
                         ids=lambda c: "n%d_s%d_p%d" % c[:3])
def test_mixed_fp32_reaches_fp64_accuracy(ctx, shape):
    """FP32 inner tGMRES + FP64 refinement reaches a true relative residual of 1e-10."""
    n, s, p, m = shape
    pr = inputs.dense_problem(n, s, p, seed=7)
    C, X, res = run(ctx, "gmres", pr, m, precision="mixed_fp32", inner_tol=1e-5)
    assert res.status == 0, res
    assert tp.norm(C - kr.sylv_apply(pr.A, pr.B, X)) <= 1e-10 * tp.norm(C)
    ref = kr.tgmres(pr.A, pr.B, C, m=m, tol=1e-10)
    assert np.abs(X - ref.X).max() <= 1e-8 * np.abs(ref.X).max()
    assert res.info.applies_low > 0 and res.info.outer >= 1


def test_fp64_full_size_n1024(ctx):
    """The 1024 x 1024 x 16 dense workload, tGMRES(30): converges to 1e-10 with the estimate
    equal to the true residual at the end of the cycle (Proposition 3.4)."""
    import torch
    cfg = inputs.WORKLOADS["dense_n1024_s1024_p16"]
    pr = inputs.dense_problem(cfg["n"], cfg["s"], cfg["p"], seed=1, scale=cfg["scale"])
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Xs = to_dev(pr.Xstar)
    Cd = ctx.sylv_apply(op, Xs)
    Xd = torch.zeros_like(Cd)
    res = ctx.tgmres_solve(op, Cd, Xd, restart=cfg["restart"], tol=1e-10)
    assert res.status == 0, res
    R = Cd - ctx.sylv_apply(op, Xd)
    assert float(torch.linalg.norm(R) / torch.linalg.norm(Cd)) <= 1e-10
    h = res.history
    assert all(b <= a * (1 + 1e-12) for a, b in zip(h, h[1:])), "GMRES estimates must not increase"
    assert abs(h[-1] - res.true_history[-1]) <= 1e-11 * res.info.normC
    err = float(torch.max(torch.abs(Xd - Xs)))
    assert err < 1e-8
    op.close()


def test_errors_are_reported(ctx):
    import torch
    from paper_2405_09233_gb300 import TstarError
    pr = inputs.dense_problem(8, 4, 3, seed=1)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    C = to_dev(inputs.random_tensor((8, 4, 3), seed=2))
    X = torch.zeros_like(C)
    with pytest.raises(TstarError) as e:
        ctx.tgmres_solve(op, C, X, restart=0)
    assert e.value.status == -1
    with pytest.raises(TstarError) as e:
        ctx.tfom_solve(op, C, X, restart=5, tol=-1.0)
    assert e.value.status == -1
    r = ctx.tgmres_solve(op, C, X, restart=2, max_restarts=1, tol=1e-14)
    assert r.status == 2                                   # budget exhausted: TS_NOT_CONVERGED
    Cn = C.clone()
    Cn[0, 0, 0] = float("nan")
    with pytest.raises(TstarError) as e:
        ctx.tgmres_solve(op, Cn, torch.zeros_like(C), restart=5)
    assert e.value.status == -4                            # TS_ERR_NONFINITE
    op.close()


@pytest.mark.parametrize("method", ["gmres", "fom"])
def test_breakdown_gives_exact_solution(ctx, method):
    """Algorithm 2's breakdown h_{j+1,j} = 0 on the GPU: M = 4 I (A^(1) = 3 I, B^(1) = -I), so C spans an
    invariant subspace, the Arnoldi process stops after one step and X = C / 4 exactly (as the oracle)."""
    import torch
    n, s, p = 4, 3, 2
    A = np.zeros((n, n, p)); A[:, :, 0] = 3.0 * np.eye(n)
    B = np.zeros((s, s, p)); B[:, :, 0] = -np.eye(s)
    C = inputs.random_tensor((n, s, p), seed=1)
    ref = kr.restarted_solve(method, A, B, C, m=5, tol=1e-10)
    assert ref.iters == 1 and ref.status == "ok"
    op = ctx.op_create_dense(to_dev(A), to_dev(B))
    Xd = torch.zeros((p, s, n), dtype=torch.float64, device="cuda")
    fn = ctx.tgmres_solve if method == "gmres" else ctx.tfom_solve
    res = fn(op, to_dev(C), Xd, restart=5, tol=1e-10)
    assert res.status == 0 and res.info.iters == 1 and res.info.cycles == 1, res
    np.testing.assert_allclose(from_dev(Xd), C / 4.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(from_dev(Xd), ref.X, rtol=0, atol=1e-15)
    op.close()
