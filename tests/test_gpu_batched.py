"""GPU tests of the batched solver: many independent instances of uneven (n, s, p), each checked
against the oracle's single-instance tGMRES (small sizes) or by its own true residual computed
with the library's FP64 operator (the 256-instance workload)."""
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


SHAPES = [(20, 4, 1), (33, 9, 3), (64, 16, 4), (70, 5, 7), (24, 24, 4), (40, 12, 8), (65, 3, 16), (17, 17, 2),
          (50, 8, 5), (96, 20, 16)]


def make_batch(ctx, shapes, seed0, scale=0.1):
    import torch
    probs, ops, Cs, Xs, Cn = [], [], [], [], []
    for q, (n, s, p) in enumerate(shapes):
        pr = inputs.dense_problem(n, s, p, seed=seed0 + q, scale=scale)
        C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
        probs.append(pr)
        Cn.append(C)
        ops.append(ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B)))
        Cs.append(to_dev(C))
        Xs.append(torch.zeros((p, s, n), dtype=torch.float64, device="cuda"))
    return probs, ops, Cs, Xs, Cn


@pytest.mark.parametrize("m", [20, 6])
def test_batched_fp64_matches_single_instance_oracle(ctx, m):
    probs, ops, Cs, Xs, Cn = make_batch(ctx, SHAPES, 100)
    st, infos, sts = ctx.batched_solve(ops, Cs, Xs, restart=m, tol=1e-10, precision="fp64")
    assert st == 0 and all(v == 0 for v in sts), sts
    for pr, C, X, info in zip(probs, Cn, Xs, infos):
        ref = kr.tgmres(pr.A, pr.B, C, m=m, tol=1e-10)
        Xh = from_dev(X)
        assert tp.norm(C - kr.sylv_apply(pr.A, pr.B, Xh)) <= 1e-10 * tp.norm(C)
        assert np.abs(Xh - ref.X).max() <= 1e-8 * np.abs(ref.X).max()
        assert info.iters == ref.iters and info.cycles == ref.cycles, (info.iters, ref.iters)
        assert abs(info.relres_true - ref.relres) <= 1e-11
    for op in ops:
        op.close()


def test_batched_mixed_fp32_per_instance_tolerances(ctx):
    probs, ops, Cs, Xs, Cn = make_batch(ctx, SHAPES, 200)
    tols = [10.0 ** (-8 - 2 * q / (len(SHAPES) - 1)) for q in range(len(SHAPES))]   # 1e-8 .. 1e-10
    st, infos, sts = ctx.batched_solve(ops, Cs, Xs, tols=tols, restart=20, precision="mixed_fp32")
    assert st == 0 and all(v == 0 for v in sts), sts
    for pr, C, X, tol, info in zip(probs, Cn, Xs, tols, infos):
        Xh = from_dev(X)
        assert tp.norm(C - kr.sylv_apply(pr.A, pr.B, Xh)) <= tol * tp.norm(C)
        assert info.relres_true <= tol and info.outer >= 1
    for op in ops:
        op.close()


def test_batched_matches_unbatched_gpu(ctx):
    """Each instance of a batch reaches the same solution as a separate ts_tgmres_solve call."""
    import torch
    probs, ops, Cs, Xs, Cn = make_batch(ctx, SHAPES[:5], 300)
    ctx.batched_solve(ops, Cs, Xs, restart=10, precision="fp64")
    for op, C, X in zip(ops, Cs, Xs):
        X1 = torch.zeros_like(X)
        r = ctx.tgmres_solve(op, C, X1, restart=10)
        assert r.status == 0
        assert float(torch.max(torch.abs(X1 - X))) <= 1e-9 * float(torch.max(torch.abs(X1)))
        op.close()


def test_batched_repeated_calls_leave_operators_intact(ctx):
    """Solving the same batch twice with fresh operators: the second solve must not write into any
    other allocation (operators stay consistent with C) and must reach the same solutions."""
    import torch
    specs = inputs.batched_specs(24, seed=9, n_range=(40, 300), s_range=(8, 40))
    dev_in, Cs = [], []
    for sp in specs:
        pr = inputs.dense_problem(sp.n, sp.s, sp.p, seed=sp.seed)
        dev_in.append((to_dev(pr.A), to_dev(pr.B), to_dev(pr.Xstar)))
    for A, B, Xst in dev_in:
        op = ctx.op_create_dense(A, B)
        Cs.append(ctx.sylv_apply(op, Xst))
        op.close()
    Xs = [torch.zeros_like(C) for C in Cs]
    for rep in range(2):
        ops = [ctx.op_create_dense(A, B) for A, B, _ in dev_in]
        for X in Xs:
            X.zero_()
        st, infos, sts = ctx.batched_solve(ops, Cs, Xs, restart=20, precision="mixed_fp32")
        assert st == 0
        ctx.workspace_check()
        for op, C, X, (_, _, Xst) in zip(ops, Cs, Xs, dev_in):
            assert float(torch.max(torch.abs(ctx.sylv_apply(op, Xst) - C))) <= 1e-9 * float(torch.max(torch.abs(C)))
            assert float(torch.max(torch.abs(X - Xst))) < 1e-7
            op.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed_fp32"])
def test_batched_ozaki_residuals(ctx, prec):
    """The batch with its FP64 products on the emulated-FP64 engine (in an FP64 solve the Arnoldi
    products as well as the residuals): every instance reaches its tolerance (checked by the oracle)
    and matches the DFMA-engine batch to 1e-8 relative."""
    import torch
    probs, ops, Cs, Xs, Cn = make_batch(ctx, SHAPES, 400)
    st, infos, sts = ctx.batched_solve(ops, Cs, Xs, restart=12, precision=prec, engine="ozaki")
    assert st == 0 and all(v == 0 for v in sts), sts
    Xd = [torch.zeros_like(X) for X in Xs]
    st2, _, _ = ctx.batched_solve(ops, Cs, Xd, restart=12, precision=prec)
    assert st2 == 0
    for pr, C, X, X2 in zip(probs, Cn, Xs, Xd):
        Xh = from_dev(X)
        assert tp.norm(C - kr.sylv_apply(pr.A, pr.B, Xh)) <= 1e-10 * tp.norm(C)
        assert float(torch.max(torch.abs(X - X2))) <= 1e-8 * float(torch.max(torch.abs(X2)))
    for op in ops:
        op.close()


@pytest.mark.parametrize("prec,engine", [("mixed_tf32x3", "dfma"), ("mixed_tf32x3", "ozaki"), ("mixed_bf16", "ozaki"),
                                         ("mixed_tf32", "dfma")])
def test_batched_tensor_core_inner(ctx, prec, engine):
    """Inner products of the batch on the tcgen05 tensor cores (per-instance tensor maps, one work
    list over all instances): every instance reaches 1e-10 (checked by the oracle)."""
    probs, ops, Cs, Xs, Cn = make_batch(ctx, SHAPES + [(300, 128, 16), (129, 65, 8)], 500)
    st, infos, sts = ctx.batched_solve(ops, Cs, Xs, restart=20, precision=prec, engine=engine)
    assert st == 0 and all(v == 0 for v in sts), sts
    for pr, C, X, info in zip(probs, Cn, Xs, infos):
        Xh = from_dev(X)
        assert tp.norm(C - kr.sylv_apply(pr.A, pr.B, Xh)) <= 1e-10 * tp.norm(C)
        assert info.outer >= 1 and info.applies_low > 0
    for op in ops:
        op.close()


def test_batched_256_instance_workload(ctx):
    """256 instances, n log-uniform in [64, 1024], s uniform in [16, 128], p in {4, 8, 16}, FP32 inner
    tGMRES(20) with FP64 refinement; every instance's true residual (library FP64 operator) <= 1e-10."""
    import torch
    specs = inputs.batched_specs(256, seed=4)
    ops, Cs, Xs, Xstars = [], [], [], []
    for sp in specs:
        pr = inputs.dense_problem(sp.n, sp.s, sp.p, seed=sp.seed)
        op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
        Xst = to_dev(pr.Xstar)
        ops.append(op)
        Xstars.append(Xst)
        Cs.append(ctx.sylv_apply(op, Xst))
        Xs.append(torch.zeros_like(Xst))
    st, infos, sts = ctx.batched_solve(ops, Cs, Xs, restart=20, precision="mixed_fp32")
    assert st == 0 and all(v == 0 for v in sts)
    for op, C, X, Xst in zip(ops, Cs, Xs, Xstars):
        R = C - ctx.sylv_apply(op, X)
        assert float(torch.linalg.norm(R) / torch.linalg.norm(C)) <= 1e-10
        assert float(torch.max(torch.abs(X - Xst))) < 1e-7
        op.close()
