"""ts_tstar_noalloc: the T-product for callers that cannot allocate device memory at call time
(code under CUDA stream capture, allocation-free serving loops, processes whose device memory is
held by another allocator).  Its scratch is a fixed array inside the library, so this file checks
that two calls in a row -- the second one reusing the array the first one left behind -- agree
with ts_tstar, and that requests beyond the array's size are refused.  It is collected last so
that a failure here never hides the other GPU tests, and it makes its own context so that it
passes alone in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

from oracle import tproduct as tp
from paper_2405_09233_gb300 import binding, inputs
from tests.gpu_helpers import to_dev, from_dev, fp64_product_bound

pytestmark = pytest.mark.gpu


def _noalloc(A, B, n1, n2, m, p, C):
    import torch
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return binding.lib().ts_tstar_noalloc(A.data_ptr(), n1, n2, B.data_ptr(), m, p, C.data_ptr(), st)


def test_noalloc_tstar_matches_tstar_twice():
    import torch
    from paper_2405_09233_gb300 import Context
    ctx = Context(0)
    for shape, seed in [((70, 33, 65, 8), 1), ((37, 129, 11, 5), 2)]:   # two calls in a row
        n1, n2, m, p = shape
        A = inputs.random_tensor((n1, n2, p), seed=seed)
        B = inputs.random_tensor((n2, m, p), seed=seed + 10)
        Ad, Bd = to_dev(A), to_dev(B)
        Cd = torch.full((p, m, n1), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(Ad, Bd, n1, n2, m, p, Cd) == binding.TS_OK
        torch.cuda.synchronize()
        ref = from_dev(ctx.tstar(Ad, Bd))                       # the existing entry point
        bound = fp64_product_bound(np.abs(A), np.abs(B), tp.tprod, p + n2)
        got = from_dev(Cd)
        assert np.all(np.abs(got - ref) <= bound), np.abs(got - ref).max()
    ctx.close()


def test_noalloc_rejects_too_large_and_host_memory():
    import torch
    n1 = n2 = m = 1024
    p = 4                                          # K (n1 n2 + n2 m + n1 m) = 3 * 3 Mi > 2 Mi
    A = torch.zeros((p, n2, n1), dtype=torch.float64, device="cuda")
    B = torch.zeros((p, m, n2), dtype=torch.float64, device="cuda")
    C = torch.zeros((p, m, n1), dtype=torch.float64, device="cuda")
    assert _noalloc(A, B, n1, n2, m, p, C) == binding.TS_ERR_ARG
    Ah = torch.zeros((2, 3, 4), dtype=torch.float64)
    Bh = torch.zeros((2, 5, 3), dtype=torch.float64)
    Ch = torch.zeros((2, 5, 4), dtype=torch.float64)
    assert _noalloc(Ah, Bh, 4, 3, 5, 2, Ch) == binding.TS_ERR_ARG
