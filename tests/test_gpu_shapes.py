"""GPU parity at the shapes where the implementation switches form, against the oracle.

Each shape sits on one side of a boundary of the CUDA path: the 8 x 4-tile slice product (reduction
lengths <= 64) against the 16/32/64 tiles; the one-launch cluster step tail (vectors <= 65536
entries, with 2, 4, 8 or 16 entries per thread) against the multi-block MGS kernels; the register
FFT (p a power of two <= 32) against the direct DFT (other p, and p > 32); the small-problem
launch-ahead cycle against the conditional cycle graph (from the second cycle on).  Residual
histories agree with the oracle's to 1e-10 ||C|| at every inner step, as in test_gpu_solvers.
"""
import numpy as np
import pytest

from oracle import krylov as kr, tproduct as tp
from paper_2405_09233_gb300 import inputs
from tests.gpu_helpers import to_dev, from_dev

pytestmark = pytest.mark.gpu

SHAPES = [  # (n, s, p, m)
    (64, 64, 3, 12),      # reduction lengths 64: 8 x 4 tiles; 12288 unknowns, 4 entries per thread
    (65, 64, 3, 12),      # n = 65: the tiled product; odd p (direct DFT)
    (64, 65, 2, 12),      # s = 65
    (32, 32, 2, 20),      # 2048 unknowns: one-CTA cluster, 2 entries per thread
    (41, 50, 4, 10),      # 8200 unknowns, ragged tiles, several cycles
    (64, 64, 16, 8),      # 65536 unknowns: the largest one-launch step tail (16 per thread)
    (65, 63, 16, 8),      # 65520 unknowns
    (33, 31, 64, 8),      # p = 64: direct DFT, 65472 unknowns
    (35, 30, 63, 8),      # 66150 unknowns: multi-block MGS and the cycle graph; odd p
    (20, 12, 33, 10),     # p = 33
]


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_09233_gb300 import Context
    c = Context(0)
    yield c
    c.workspace_check()
    c.close()


@pytest.mark.parametrize("method", ["gmres", "fom"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda c: "n%d_s%d_p%d_m%d" % c)
def test_boundary_shapes_match_oracle(ctx, method, shape):
    import torch
    n, s, p, m = shape
    pr = inputs.dense_problem(n, s, p, seed=300 + n + 7 * p)
    C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Xd = to_dev(np.zeros_like(C))
    fn = ctx.tgmres_solve if method == "gmres" else ctx.tfom_solve
    res = fn(op, to_dev(C), Xd, restart=m, tol=1e-10)
    torch.cuda.synchronize()
    X = from_dev(Xd)
    op.close()
    ref = kr.restarted_solve(method, pr.A, pr.B, C, m=m, tol=1e-10)
    assert res.status == 0 and ref.status == "ok"
    assert len(res.history) == len(ref.history), (len(res.history), len(ref.history))
    np.testing.assert_allclose(res.history, ref.history, rtol=0, atol=1e-10 * ref.normC)
    assert res.info.cycles == ref.cycles
    assert tp.norm(C - kr.sylv_apply(pr.A, pr.B, X)) <= 1e-10 * tp.norm(C)


@pytest.mark.parametrize("shape", [(64, 64, 3), (65, 64, 3), (33, 31, 64), (96, 40, 6)],
                         ids=lambda c: "n%d_s%d_p%d" % c)
def test_boundary_shapes_apply_matches_oracle(ctx, shape):
    """M(X) itself at the product-tile and DFT boundaries, entry by entry against Definition 2.1."""
    n, s, p = shape
    pr = inputs.dense_problem(n, s, p, seed=400 + n)
    X = inputs.random_tensor((n, s, p), seed=401)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Y = from_dev(ctx.sylv_apply(op, to_dev(X)))
    op.close()
    ref = kr.sylv_apply(pr.A, pr.B, X)
    np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
