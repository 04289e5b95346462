"""GPU parity of the emulated-FP64 tensor-core engine (Ozaki scheme) against the oracle, through the
C ABI: the operator itself, and tGMRES / tFOM / mixed-precision refinement running on it.

Tolerance of the emulated operator.  Per Fourier slice k, with alpha_k = 2^E_op (max |Re|, |Im| of
A_k and B_k below alpha_k / 2) and xi_k = 2^E_x (likewise for X_k), each of the L = n + s terms of
an entry of A_k X_k - X_k B_k carries the digit truncation of both factors (2 alpha_k xi_k 2^(-8S-1))
and the dropped digit pairs (< (S - 1) alpha_k xi_k 2^(-8S-1)); the fixed-point roundings are
below 2^-60 alpha_k xi_k L.  The inverse DFT averages the slices, so every entry of M(X) is within
    L max_k alpha_k xi_k 2^(-8S) (S + 1) / 2
of the exactly rounded slice products, on top of the FP64 rounding bound of the DFT route (the
same one the DFMA engine is held to).  The test applies that sum with a factor 2 of margin.
"""
import numpy as np
import pytest

from oracle import krylov as kr, tproduct as tp
from paper_2405_09233_gb300 import inputs
from tests.gpu_helpers import to_dev, from_dev, fp64_product_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_09233_gb300 import Context
    c = Context(0)
    yield c
    c.workspace_check()          # no kernel wrote past the end of a workspace buffer
    c.close()


def slice_scale(T3):
    """2^E per Fourier slice k <= p/2 with max(|Re|, |Im|) < 2^(E-1), as the engine chooses E."""
    F = np.fft.fft(T3, axis=2)[:, :, : T3.shape[2] // 2 + 1]
    m = np.maximum(np.abs(F.real), np.abs(F.imag)).max(axis=(0, 1))
    return np.where(m > 0, 2.0 ** (np.floor(np.log2(np.where(m > 0, m, 1.0))) + 2), 0.0), m


def ozaki_bound(A, B, X, S):
    n, s, p = X.shape
    a_ab = np.maximum(slice_scale(A)[1], slice_scale(B)[1])
    alpha = np.where(a_ab > 0, 2.0 ** (np.floor(np.log2(np.where(a_ab > 0, a_ab, 1.0))) + 2), 0.0)
    xi = slice_scale(X)[0]
    return 2.0 * (n + s) * np.max(alpha * xi) * 2.0 ** (-8 * S) * (S + 1) / 2


SHAPES = [(1, 1, 1), (24, 24, 4), (37, 5, 7), (65, 63, 8), (130, 70, 16), (100, 3, 2), (8, 70, 16),
          (200, 130, 32), (10, 6, 33), (129, 257, 3)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_ozaki_apply_matches_oracle(ctx, shape):
    n, s, p = shape
    pr = inputs.dense_problem(n, s, p, seed=3 + n)
    X = inputs.random_tensor((n, s, p), seed=5)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Y = from_dev(ctx.sylv_apply_ozaki(op, to_dev(X)))
    ref = kr.sylv_apply(pr.A, pr.B, X)
    bound = (fp64_product_bound(np.abs(pr.A), np.abs(X), tp.tprod, p + n)
             + fp64_product_bound(np.abs(X), np.abs(pr.B), tp.tprod, p + s)
             + ozaki_bound(pr.A, pr.B, X, 6))
    err = np.abs(Y - ref)
    assert np.all(err <= bound), (err / bound).max()
    op.close()


@pytest.mark.parametrize("digits", [3, 4, 5, 7, 8])
def test_ozaki_digit_counts(ctx, digits):
    """Fewer digits: larger error, still inside the bound; the error shrinks as digits are added
    until the FP64 rounding of the DFTs dominates."""
    n, s, p = 96, 40, 8
    pr = inputs.dense_problem(n, s, p, seed=11)
    X = inputs.random_tensor((n, s, p), seed=12)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Y = from_dev(ctx.sylv_apply_ozaki(op, to_dev(X), digits=digits))
    ref = kr.sylv_apply(pr.A, pr.B, X)
    bound = (fp64_product_bound(np.abs(pr.A), np.abs(X), tp.tprod, p + n)
             + fp64_product_bound(np.abs(X), np.abs(pr.B), tp.tprod, p + s)
             + ozaki_bound(pr.A, pr.B, X, digits))
    err = np.abs(Y - ref)
    assert np.all(err <= bound), (err / bound).max()
    if digits == 3:
        assert err.max() > 1e-9 * np.abs(ref).max()      # 3 digits (23 bits) cannot reach FP64 level
    op.close()


@pytest.mark.parametrize("digits", [3, 4, 5])
def test_ozaki_leading_digits(ctx, digits):
    """An operator prepared with 8 digits, applied through its leading 3..5: inside the same bound
    as an expansion with that many digits, and bit-identical to a second call."""
    n, s, p = 96, 40, 8
    pr = inputs.dense_problem(n, s, p, seed=11)
    X = inputs.random_tensor((n, s, p), seed=12)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    ctx.sylv_apply_ozaki(op, to_dev(X), digits=8)                 # digit planes built with 8 digits
    Y = from_dev(ctx.sylv_apply_ozaki(op, to_dev(X), digits=digits))
    ref = kr.sylv_apply(pr.A, pr.B, X)
    bound = (fp64_product_bound(np.abs(pr.A), np.abs(X), tp.tprod, p + n)
             + fp64_product_bound(np.abs(X), np.abs(pr.B), tp.tprod, p + s)
             + ozaki_bound(pr.A, pr.B, X, digits))
    err = np.abs(Y - ref)
    assert np.all(err <= bound), (err / bound).max()
    Y8 = from_dev(ctx.sylv_apply_ozaki(op, to_dev(X), digits=8))   # full digits again afterwards
    assert np.all(np.abs(Y8 - ref) <= bound)
    assert np.abs(Y8 - ref).max() < err.max() or digits >= 5
    assert np.array_equal(Y, from_dev(ctx.sylv_apply_ozaki(op, to_dev(X), digits=digits)))
    op.close()


def test_mixed_ozaki_progressive_digits(ctx):
    """BF16 inner solve, emulated residuals with progressive digits (default) and with 6 fixed
    digits: both reach 1e-10 (oracle check), with the same number of outer steps within one, and a
    later full-digit application is unaffected."""
    n, s, p, m = 200, 130, 8, 20
    pr = inputs.dense_problem(n, s, p, seed=21)
    C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    outs = {}
    for digits in (0, 6):
        Xd = to_dev(np.zeros_like(C))
        res = ctx.tgmres_solve(op, to_dev(C), Xd, restart=m, tol=1e-10, precision="mixed_bf16", engine="ozaki",
                               ozaki_digits=digits)
        assert res.status == 0, res
        X = from_dev(Xd)
        assert tp.norm(C - kr.sylv_apply(pr.A, pr.B, X)) <= 1e-10 * tp.norm(C)
        outs[digits] = res.info.outer
    assert abs(outs[0] - outs[6]) <= 1, outs
    Xr = inputs.random_tensor((n, s, p), seed=5)
    Y = from_dev(ctx.sylv_apply_ozaki(op, to_dev(Xr)))
    ref = kr.sylv_apply(pr.A, pr.B, Xr)
    bound = (fp64_product_bound(np.abs(pr.A), np.abs(Xr), tp.tprod, p + n)
             + fp64_product_bound(np.abs(Xr), np.abs(pr.B), tp.tprod, p + s)
             + ozaki_bound(pr.A, pr.B, Xr, 6))
    assert np.all(np.abs(Y - ref) <= bound)
    op.close()


def test_ozaki_scaled_operands(ctx):
    """Operands far from unit magnitude (A, B scaled by 2^40, X by 2^-70): the per-slice exponents
    absorb the scaling."""
    n, s, p = 70, 33, 6
    pr = inputs.dense_problem(n, s, p, seed=21)
    A, B = pr.A * 2.0 ** 40, pr.B * 2.0 ** 40
    X = inputs.random_tensor((n, s, p), seed=22) * 2.0 ** -70
    op = ctx.op_create_dense(to_dev(A), to_dev(B))
    Y = from_dev(ctx.sylv_apply_ozaki(op, to_dev(X)))
    ref = kr.sylv_apply(A, B, X)
    bound = (fp64_product_bound(np.abs(A), np.abs(X), tp.tprod, p + n)
             + fp64_product_bound(np.abs(X), np.abs(B), tp.tprod, p + s) + ozaki_bound(A, B, X, 6))
    assert np.all(np.abs(Y - ref) <= bound)
    op.close()


def test_ozaki_zero_and_nonfinite(ctx):
    import torch
    pr = inputs.dense_problem(20, 6, 4, seed=1)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Z = torch.zeros((4, 6, 20), dtype=torch.float64, device="cuda")
    assert float(torch.max(torch.abs(ctx.sylv_apply_ozaki(op, Z)))) == 0.0
    Xn = to_dev(inputs.random_tensor((20, 6, 4), seed=2))
    Xn[1, 2, 3] = float("nan")
    assert not bool(torch.isfinite(ctx.sylv_apply_ozaki(op, Xn)).all())
    op.close()


def test_ozaki_full_size_sampled(ctx):
    """The 1024 x 1024 x 16 dense workload on the emulated engine: sampled entries against the
    oracle's single-entry Definition 2.1, within the FP64 entry bound plus the engine's term."""
    cfg = inputs.WORKLOADS["dense_n1024_s1024_p16"]
    pr = inputs.dense_problem(cfg["n"], cfg["s"], cfg["p"], seed=1, scale=cfg["scale"])
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Y = from_dev(ctx.sylv_apply_ozaki(op, to_dev(pr.Xstar)))
    n, s, p = pr.Xstar.shape
    extra = ozaki_bound(pr.A, pr.B, pr.Xstar, 6)
    rng = np.random.default_rng(2)
    idx = [(0, 0, 0), (n - 1, s - 1, p - 1)] + [tuple(int(rng.integers(d)) for d in (n, s, p)) for _ in range(40)]
    for (i, j, k) in idx:
        ref = tp.tentry(pr.A, pr.Xstar, i, j, k) - tp.tentry(pr.Xstar, pr.B, i, j, k)
        mag = tp.tentry(np.abs(pr.A), np.abs(pr.Xstar), i, j, k) + tp.tentry(np.abs(pr.Xstar), np.abs(pr.B), i, j, k)
        assert abs(Y[i, j, k] - ref) <= 8 * (p + n) * 2.0 ** -53 * mag + extra, (i, j, k)
    op.close()


CASES = [(24, 24, 4, 20, 0), (24, 24, 4, 5, 0), (37, 5, 7, 8, 3), (16, 9, 1, 10, 4), (70, 66, 16, 12, 5)]


@pytest.mark.parametrize("method", ["gmres", "fom"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "n%d_s%d_p%d_m%d" % c[:4])
@pytest.mark.parametrize("spectral", [False, True], ids=["real_basis", "spectral_basis"])
def test_ozaki_solve_history_parity(ctx, method, case, spectral):
    """tGMRES / tFOM with every FP64 application on the emulated engine: the residual history
    matches the oracle's to 1e-10 ||C|| at every inner step, as the DFMA engine's does, with the
    Krylov basis in real space or in the Fourier domain."""
    n, s, p, m, seed = case
    pr = inputs.dense_problem(n, s, p, seed=seed)
    C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Xd = to_dev(np.zeros_like(C))
    fn = ctx.tgmres_solve if method == "gmres" else ctx.tfom_solve
    res = fn(op, to_dev(C), Xd, restart=m, tol=1e-10, engine="ozaki", spectral=spectral)
    X = from_dev(Xd)
    ref = kr.restarted_solve(method, pr.A, pr.B, C, m=m, tol=1e-10)
    assert res.status == 0 and ref.status == "ok"
    assert len(res.history) == len(ref.history)
    np.testing.assert_allclose(res.history, ref.history, rtol=0, atol=1e-10 * ref.normC)
    np.testing.assert_allclose(res.true_history, ref.true_res, rtol=0, atol=1e-10 * ref.normC)
    assert tp.norm(C - kr.sylv_apply(pr.A, pr.B, X)) <= 1e-10 * tp.norm(C)
    assert np.abs(X - ref.X).max() <= 1e-8 * np.abs(ref.X).max()
    op.close()


@pytest.mark.parametrize("prec", ["mixed_fp32", "mixed_tf32x3", "mixed_bf16"])
def test_mixed_with_ozaki_residuals(ctx, prec):
    """Mixed-precision refinement whose FP64 true residuals run on the emulated engine still
    reaches a true relative residual of 1e-10 (checked by the oracle)."""
    n, s, p, m = 130, 70, 8, 20
    pr = inputs.dense_problem(n, s, p, seed=7)
    C = kr.sylv_apply(pr.A, pr.B, pr.Xstar)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Xd = to_dev(np.zeros_like(C))
    res = ctx.tgmres_solve(op, to_dev(C), Xd, restart=m, tol=1e-10, precision=prec, engine="ozaki")
    X = from_dev(Xd)
    assert res.status == 0, res
    assert tp.norm(C - kr.sylv_apply(pr.A, pr.B, X)) <= 1e-10 * tp.norm(C)
    op.close()


def test_mixed_ozaki_full_size_n4096(ctx):
    """The 4096 x 256 x 32 workload: split-TF32 inner tGMRES(40), emulated FP64 residuals; the
    final true residual is re-checked with the DFMA engine."""
    import torch
    cfg = inputs.WORKLOADS["dense_n4096_s256_p32_g0.3"]
    pr = inputs.dense_problem(cfg["n"], cfg["s"], cfg["p"], seed=1, scale=cfg["scale"])
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Xs = to_dev(pr.Xstar)
    Cd = ctx.sylv_apply(op, Xs)
    Xd = torch.zeros_like(Cd)
    res = ctx.tgmres_solve(op, Cd, Xd, restart=cfg["restart"], tol=1e-10, precision="mixed_tf32x3", engine="ozaki")
    assert res.status == 0, res
    R = Cd - ctx.sylv_apply(op, Xd)
    assert float(torch.linalg.norm(R) / torch.linalg.norm(Cd)) <= 1e-10
    assert float(torch.max(torch.abs(Xd - Xs))) < 1e-8
    op.close()


def test_ozaki_argument_errors(ctx):
    from paper_2405_09233_gb300 import TstarError
    pr = inputs.dense_problem(8, 4, 3, seed=1)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    X = to_dev(inputs.random_tensor((8, 4, 3), seed=2))
    with pytest.raises(TstarError) as e:
        ctx.sylv_apply_ozaki(op, X, digits=2)
    assert e.value.status == -1
    with pytest.raises(TstarError) as e:
        ctx.tgmres_solve(op, X, X.clone() * 0, engine=7)
    assert e.value.status == -1
    op.close()
