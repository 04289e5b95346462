"""GPU parity of the low-precision operators (FP32 CUDA cores, TF32 and BF16 tcgen05 tensor cores)
against the FP64 oracle, and mixed-precision solves that must still reach a true relative residual
of 1e-10.

Tolerance of the low-precision operator.  The Fourier slices obey |A_k(i,l)| <= Abar(i,l) =
sum_t |A(i,l,t)| (and likewise for X and B).  Rounding each input of a slice product to a format
with unit roundoff u (2^-9 for BF16, 2^-12 for TF32, 2^-25 for FP32) perturbs each product term by
at most ~2u of its magnitude, FP32 accumulation over L terms adds L * 2^-24, and the inverse DFT
averages, so every entry of M(X) is within
    4 (2u + (n + s + p) 2^-24) (Abar Xbar + Xbar Bbar)(i, j)
of the exact value (a factor 2 of margin on top of the first-order bound).
"""
import numpy as np
import pytest

from oracle import krylov as kr, tproduct as tp
from paper_2405_09233_gb300 import inputs
from tests.gpu_helpers import to_dev, from_dev

pytestmark = pytest.mark.gpu

# split TF32 represents each input as hi + lo to ~22 bits; the dropped lo*lo term is of the same size
U = {"mixed_fp32": 2.0 ** -25, "mixed_tf32": 2.0 ** -12, "mixed_bf16": 2.0 ** -9, "mixed_tf32x3": 2.0 ** -21}


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_09233_gb300 import Context
    c = Context(0)
    yield c
    c.workspace_check()          # no kernel wrote past the end of a workspace buffer
    c.close()


SHAPES = [(24, 24, 4), (37, 5, 7), (130, 70, 8), (256, 64, 16), (200, 130, 32), (64, 256, 2), (16, 9, 1),
          (129, 257, 3)]


@pytest.mark.parametrize("prec", ["mixed_fp32", "mixed_tf32", "mixed_bf16", "mixed_tf32x3"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_lowp_apply_matches_oracle(ctx, prec, shape):
    import torch
    n, s, p = shape
    pr = inputs.dense_problem(n, s, p, seed=2 + n)
    X32 = inputs.random_tensor((n, s, p), seed=3).astype(np.float32)
    X = X32.astype(np.float64)                       # the exact input the GPU sees
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Xd = torch.from_numpy(inputs.to_device_layout(X32)).cuda()
    Y = from_dev(ctx.sylv_apply_lowp(op, Xd, prec)).astype(np.float64)
    ref = kr.sylv_apply(pr.A, pr.B, X)
    Ab, Bb, Xb = (np.abs(T).sum(axis=2) for T in (pr.A, pr.B, X))
    mag = Ab @ Xb + Xb @ Bb
    bound = 4.0 * (2 * U[prec] + (n + s + p) * 2.0 ** -24) * mag[:, :, None]
    err = np.abs(Y - ref)
    assert np.all(err <= bound), (err / bound).max()
    rel = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
    assert rel < {"mixed_fp32": 1e-5, "mixed_tf32": 3e-3, "mixed_bf16": 2e-2, "mixed_tf32x3": 1e-5}[prec], rel
    op.close()


@pytest.mark.parametrize("prec,inner", [("mixed_tf32", 1e-3), ("mixed_bf16", 1e-2), ("mixed_tf32x3", 1e-6)])
@pytest.mark.parametrize("shape", [(24, 24, 4, 20), (130, 70, 8, 20), (256, 64, 16, 30)],
                         ids=lambda c: "n%d_s%d_p%d" % c[:3])
def test_mixed_tensor_core_reaches_fp64_accuracy(ctx, prec, inner, shape):
    import torch
    n, s, p, m = shape
    pr = inputs.dense_problem(n, s, p, seed=7)
    C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Xd = torch.zeros((p, s, n), dtype=torch.float64, device="cuda")
    res = ctx.tgmres_solve(op, to_dev(C), Xd, restart=m, tol=1e-10, precision=prec, inner_tol=inner)
    X = from_dev(Xd)
    assert res.status == 0, res
    assert tp.norm(C - kr.sylv_apply(pr.A, pr.B, X)) <= 1e-10 * tp.norm(C)
    ref = kr.tgmres(pr.A, pr.B, C, m=m, tol=1e-10)
    assert np.abs(X - ref.X).max() <= 1e-8 * np.abs(ref.X).max()
    op.close()


@pytest.mark.parametrize("prec", ["mixed_bf16", "mixed_tf32", "mixed_fp32", "mixed_tf32x3"])
def test_mixed_full_size_n4096_s256_p32(ctx, prec):
    """The 4096 x 256 x 32 mixed-precision workload (perturbation 0.3): FP64 refinement around a
    low-precision tGMRES(40) reaches a true relative residual of 1e-10 (checked with the FP64
    operator, itself pinned by test_gpu_apply's sampled full-size check)."""
    import torch
    cfg = inputs.WORKLOADS["dense_n4096_s256_p32_g0.3"]
    pr = inputs.dense_problem(cfg["n"], cfg["s"], cfg["p"], seed=1, scale=cfg["scale"])
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Xs = to_dev(pr.Xstar)
    Cd = ctx.sylv_apply(op, Xs)
    Xd = torch.zeros_like(Cd)
    res = ctx.tgmres_solve(op, Cd, Xd, restart=cfg["restart"], tol=1e-10, precision=prec)
    assert res.status == 0, res
    R = Cd - ctx.sylv_apply(op, Xd)
    assert float(torch.linalg.norm(R) / torch.linalg.norm(Cd)) <= 1e-10
    assert float(torch.max(torch.abs(Xd - Xs))) < 1e-8
    op.close()


def test_lowp_rejects_host_memory(ctx):
    import torch
    from paper_2405_09233_gb300 import binding
    pr = inputs.dense_problem(8, 4, 2, seed=1)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Xh = torch.zeros((2, 4, 8), dtype=torch.float32)
    Yh = torch.zeros_like(Xh)
    st = binding.lib().ts_sylv_apply_lowp(ctx._h, op._h, 3, Xh.data_ptr(), Yh.data_ptr(), None)
    assert st == binding.TS_ERR_ARG
    op.close()
