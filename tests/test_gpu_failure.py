"""Failure detection on the GPU without a fault: a bounded device-side wait that runs out.

The tcgen05 kernels bound every mbarrier wait by elapsed time.  With TSTAR_TEST_STALL_TMA=1 in the
environment the TMA producer of the single-instance tensor-core product arms no stage (it issues no
load at all), so the MMA warp's wait on a stage that nothing fills expires after 50 ms; the kernel
records the error, frees its tensor memory and returns, and the mixed-precision solve reports
TS_ERR_TIMEOUT.  No copy or MMA is left in flight, nothing faults, and the same context must then
solve normally (which also shows the tensor memory was released: every later kernel allocates it).
"""
import pytest

from oracle import krylov as kr, tproduct as tp
from paper_2405_09233_gb300 import inputs
from tests.gpu_helpers import to_dev, from_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["mixed_bf16", "mixed_tf32x3"])
def test_expired_wait_reports_timeout_and_context_survives(monkeypatch, precision):
    import torch
    from paper_2405_09233_gb300 import Context, TstarError
    ctx = Context(0)
    pr = inputs.dense_problem(96, 40, 4, seed=3)
    C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Cd = to_dev(C)
    X = torch.zeros_like(Cd)
    monkeypatch.setenv("TSTAR_TEST_STALL_TMA", "1")
    with pytest.raises(TstarError) as e:
        ctx.tgmres_solve(op, Cd, X, restart=3, tol=1e-10, precision=precision, max_outer=1)
    assert e.value.status == -5, e.value          # TS_ERR_TIMEOUT
    monkeypatch.delenv("TSTAR_TEST_STALL_TMA")
    X.zero_()
    res = ctx.tgmres_solve(op, Cd, X, restart=20, tol=1e-10, precision=precision)
    assert res.status == 0, res
    assert tp.norm(C - kr.sylv_apply(pr.A, pr.B, from_dev(X))) <= 1e-10 * tp.norm(C)
    op.close()
    ctx.workspace_check()
    ctx.close()
