"""ts_tstar_noalloc: the T-product for callers that cannot allocate device memory when they need one
(allocation-free serving loops, processes whose device memory another allocator already holds).
Its scratch is a fixed array inside the library, so this file checks that calls in a row -- each
reusing the array the previous one left behind -- agree with the oracle's Definition 2.1 and with
ts_tstar, that a request of exactly the array's size is served and one entry more is refused, and
that memory the kernels must not be given is refused before any launch.  It is collected last so that
a failure here never hides the other GPU tests, and it makes its own context so that it passes alone
in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

from oracle import tproduct as tp
from paper_2405_09233_gb300 import binding, inputs
from tests.gpu_helpers import to_dev, from_dev, fp64_product_bound

pytestmark = pytest.mark.gpu

MAX_COMPLEX = 2 * 1024 * 1024          # TS_NOALLOC_MAX_COMPLEX


def _noalloc(A, B, n1, n2, m, p, C):
    import torch
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return binding.lib().ts_tstar_noalloc(A.data_ptr(), n1, n2, B.data_ptr(), m, p, C.data_ptr(), st)


def _check(ctx, shape, seed):
    import torch
    n1, n2, m, p = shape
    A = inputs.random_tensor((n1, n2, p), seed=seed)
    B = inputs.random_tensor((n2, m, p), seed=seed + 10)
    Ad, Bd = to_dev(A), to_dev(B)
    Cd = torch.full((p, m, n1), float("nan"), dtype=torch.float64, device="cuda")
    assert _noalloc(Ad, Bd, n1, n2, m, p, Cd) == binding.TS_OK
    torch.cuda.synchronize()
    got = from_dev(Cd)
    bound = fp64_product_bound(np.abs(A), np.abs(B), tp.tprod, p + n2)
    ref = tp.tprod(A, B)                                    # the oracle (Definition 2.1)
    assert np.all(np.abs(got - ref) <= bound), np.abs(got - ref).max()
    assert np.all(np.abs(got - from_dev(ctx.tstar(Ad, Bd))) <= bound)   # and the allocating entry point


def test_noalloc_tstar_matches_oracle_calls_in_a_row():
    from paper_2405_09233_gb300 import Context
    ctx = Context(0)
    # several calls in a row, each over what the previous one left in the scratch array:
    # p = 8 (even, two tiles in each direction), odd p = 5, p = 1 (a matrix product), odd p = 33 > 32
    for shape, seed in [((70, 33, 65, 8), 1), ((37, 129, 11, 5), 2), ((50, 20, 30, 1), 3), ((9, 7, 5, 33), 4),
                        ((70, 33, 65, 8), 5)]:
        _check(ctx, shape, seed)
    ctx.close()


def test_noalloc_size_limit_is_exact():
    """K (n1 n2 + n2 m + n1 m) == TS_NOALLOC_MAX_COMPLEX is served; one more complex entry is refused."""
    import torch
    from paper_2405_09233_gb300 import Context
    ctx = Context(0)
    for p, n1 in [(1, 524287), (3, 262143)]:           # K = 1: 4 n1 + 4 = 2 Mi; K = 2: 2 (4 n1 + 4) = 2 Mi
        K = p // 2 + 1
        assert K * (n1 * 2 + 2 * 2 + n1 * 2) == MAX_COMPLEX
        _check(ctx, (n1, 2, 2, p), seed=p)
        A = torch.zeros((p, 2, n1 + 1), dtype=torch.float64, device="cuda")
        B = torch.zeros((p, 2, 2), dtype=torch.float64, device="cuda")
        C = torch.zeros((p, 2, n1 + 1), dtype=torch.float64, device="cuda")
        assert K * ((n1 + 1) * 2 + 4 + (n1 + 1) * 2) > MAX_COMPLEX
        assert _noalloc(A, B, n1 + 1, 2, 2, p, C) == binding.TS_ERR_ARG
    ctx.close()


def test_noalloc_rejects_host_and_other_device_memory():
    """Memory the kernels must not be given is refused (TS_ERR_ARG) before anything is launched."""
    import torch
    Ah = torch.zeros((2, 3, 4), dtype=torch.float64)
    Bh = torch.zeros((2, 5, 3), dtype=torch.float64)
    Ch = torch.zeros((2, 5, 4), dtype=torch.float64)
    assert _noalloc(Ah, Bh, 4, 3, 5, 2, Ch) == binding.TS_ERR_ARG
    n1 = n2 = m = 1024
    p = 4                                          # K (n1 n2 + n2 m + n1 m) = 3 * 3 Mi > 2 Mi
    A = torch.zeros((p, n2, n1), dtype=torch.float64, device="cuda")
    B = torch.zeros((p, m, n2), dtype=torch.float64, device="cuda")
    C = torch.zeros((p, m, n1), dtype=torch.float64, device="cuda")
    assert _noalloc(A, B, n1, n2, m, p, C) == binding.TS_ERR_ARG
    if torch.cuda.device_count() < 2:
        pytest.skip("one GPU: the other-device case needs two")
    A1 = torch.zeros((2, 3, 4), dtype=torch.float64, device="cuda:1")
    B0 = torch.zeros((2, 5, 3), dtype=torch.float64, device="cuda:0")
    C0 = torch.zeros((2, 5, 4), dtype=torch.float64, device="cuda:0")
    with torch.cuda.device(0):
        assert _noalloc(A1, B0, 4, 3, 5, 2, C0) == binding.TS_ERR_ARG
