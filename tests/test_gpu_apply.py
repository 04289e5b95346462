"""GPU parity of the T-product and of the Sylvester operator against the oracle (through the C ABI)."""
import numpy as np
import pytest

from oracle import tproduct as tp, krylov as kr
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


TSTAR_SHAPES = [  # (n1, n2, m, p): ragged sizes, several 64-tiles, odd/even p, p = 1, p beyond the unrolled range
    (1, 1, 1, 1), (3, 2, 4, 1), (5, 7, 3, 2), (65, 33, 17, 3), (130, 70, 129, 4), (64, 64, 64, 5),
    (37, 129, 11, 7), (20, 9, 66, 8), (71, 40, 3, 16), (9, 8, 7, 17), (33, 31, 29, 32), (6, 5, 4, 33),
    (12, 10, 8, 64), (5, 4, 3, 70),
]


@pytest.mark.parametrize("shape", TSTAR_SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_tstar_matches_oracle(ctx, shape):
    n1, n2, m, p = shape
    A = inputs.random_tensor((n1, n2, p), seed=n1 + 7 * p)
    B = inputs.random_tensor((n2, m, p), seed=m + 11 * p)
    C = from_dev(ctx.tstar(to_dev(A), to_dev(B)))
    ref = tp.tprod(A, B)
    bound = fp64_product_bound(np.abs(A), np.abs(B), tp.tprod, p + n2)
    assert np.all(np.abs(C - ref) <= bound), np.abs(C - ref).max()


def test_tstar_host_buffers(ctx):
    """Host (CPU) tensors go through the same C-ABI call and give the same bytes as device tensors."""
    A = inputs.random_tensor((40, 30, 6), seed=1)
    B = inputs.random_tensor((30, 20, 6), seed=2)
    Cd = from_dev(ctx.tstar(to_dev(A), to_dev(B)))
    Ch = from_dev(ctx.tstar(to_dev(A, "cpu"), to_dev(B, "cpu")))
    np.testing.assert_array_equal(Cd, Ch)


APPLY_SHAPES = [(1, 1, 1), (24, 24, 4), (37, 5, 7), (65, 63, 8), (100, 3, 2), (8, 70, 16), (130, 17, 32), (10, 6, 33)]


@pytest.mark.parametrize("shape", APPLY_SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_sylv_apply_matches_oracle(ctx, shape):
    n, s, p = shape
    pr = inputs.dense_problem(n, s, p, seed=3 + n)
    X = inputs.random_tensor((n, s, p), seed=5)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Y = from_dev(ctx.sylv_apply(op, to_dev(X)))
    ref = kr.sylv_apply(pr.A, pr.B, X)
    bound = (fp64_product_bound(np.abs(pr.A), np.abs(X), tp.tprod, p + n)
             + fp64_product_bound(np.abs(X), np.abs(pr.B), tp.tprod, p + s))
    assert np.all(np.abs(Y - ref) <= bound), np.abs(Y - ref).max()
    op.close()


def sampled_apply_check(A, B, X, Y, n_samples, seed):
    """Check sampled entries of Y = M(X) against the oracle's single-entry Definition 2.1."""
    n, s, p = X.shape
    rng = np.random.default_rng(seed)
    idx = [(0, 0, 0), (n - 1, s - 1, p - 1)] + [tuple(int(rng.integers(d)) for d in (n, s, p))
                                                for _ in range(n_samples)]
    for (i, j, k) in idx:
        ref = tp.tentry(A, X, i, j, k) - tp.tentry(X, B, i, j, k)
        mag = (tp.tentry(np.abs(A), np.abs(X), i, j, k) + tp.tentry(np.abs(X), np.abs(B), i, j, k))
        assert abs(Y[i, j, k] - ref) <= 8 * (p + n) * 2.0 ** -53 * mag, (i, j, k, Y[i, j, k], ref)


@pytest.mark.parametrize("wl", ["dense_n1024_s1024_p16", "dense_n4096_s256_p32_g0.3"])
def test_sylv_apply_full_size_sampled(ctx, wl):
    """The full-size dense workloads, in the launch configuration the solver uses: sampled entries."""
    cfg = inputs.WORKLOADS[wl]
    pr = inputs.dense_problem(cfg["n"], cfg["s"], cfg["p"], seed=1, scale=cfg["scale"])
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Xd = to_dev(pr.Xstar)
    Y = from_dev(ctx.sylv_apply(op, Xd))
    sampled_apply_check(pr.A, pr.B, pr.Xstar, Y, 40, seed=2)
    op.close()


def test_sylv_apply_host_buffers_and_errors(ctx):
    from paper_2405_09233_gb300 import TstarError
    pr = inputs.dense_problem(20, 6, 5, seed=9)
    X = inputs.random_tensor((20, 6, 5), seed=1)
    op = ctx.op_create_dense(to_dev(pr.A, "cpu"), to_dev(pr.B, "cpu"))
    Yh = from_dev(ctx.sylv_apply(op, to_dev(X, "cpu")))
    Yd = from_dev(ctx.sylv_apply(op, to_dev(X)))
    np.testing.assert_array_equal(Yh, Yd)
    Xd = to_dev(X)
    with pytest.raises(TstarError) as e:
        ctx.sylv_apply(op, Xd, Xd)          # aliasing output is rejected
    assert e.value.status == -1
    op.close()
