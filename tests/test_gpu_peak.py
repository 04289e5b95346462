"""The measured FP64 roof (ts_probe_fp64_peak), the cross-check the bench reports beside the roof derived
from unit counts: GB300 issues 2 FP64 fused multiply-adds per clock per SM, 1.26 TFLOP/s at 152 SMs and
2.07 GHz, and the FP64 slice products execute ~1.18 TFLOP/s of it, so the loop's rate lies between."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp64_probe_rate_is_plausible():
    from paper_2405_09233_gb300 import Context
    with Context(0) as ctx:
        t1 = ctx.probe_fp64_peak()
        t2 = ctx.probe_fp64_peak()
        ctx.workspace_check()
    for t in (t1, t2):
        assert 0.5 < t < 2.0, t
    assert abs(t1 - t2) <= 0.1 * max(t1, t2), (t1, t2)
