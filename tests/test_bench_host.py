"""Host logic of bench.py (no GPU): roofline arithmetic, measured-traffic lookup, peaks source."""
import json
import os

import pytest

import bench


def test_traffic_only_for_the_captured_workload():
    assert bench.traffic_for("k_gemm_slices<double>", "dense_n1024_s1024_p16") == 497799168 + 137544960
    assert bench.traffic_for("k_oz_sylv/6", "dense_n1024_s1024_p16") == 1779147520 + 149931264
    assert bench.traffic_for("k_gemm_slices<double>", "dense_n4096_s256_p32_g0.3") is None
    assert bench.traffic_for("k_tc_sylv", "dense_n1024_s1024_p16") is None


def test_ozaki_roofline_counts_the_issued_digit_pairs():
    pk = bench.peaks()
    flops, ms = 128.8e9, 3.0
    r6 = bench.ozaki_roofline(flops, 21 * flops, ms, True, 0.5)
    assert r6["achieved"] == pytest.approx(21 * flops / (ms * 1e-3) / 1e12)
    assert r6["peak"] == pk["bf16_sustained"]
    assert r6["frac"] == pytest.approx(r6["achieved"] / r6["peak"])
    assert "21.0 BF16 digit-pair" in r6["kernel"]
    # a mixed solve whose launches used 4, 5 and 6 digits: 10 + 15 + 21 pairs over three launches
    r = bench.ozaki_roofline(flops, (10 + 15 + 21) * flops / 3, ms, False, 0.4)
    assert r["peak"] == pk["bf16_burst"]
    assert "15.3 BF16 digit-pair" in r["kernel"]


def test_gemm_roofline_fp64_and_tensor_peaks():
    r = bench.gemm_roofline("fp64", "fp64", 128.8e9, 84.0, True, 0.98)
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(4 * 152 * 2.070e9 / 1e12)
    assert r["achieved"] == pytest.approx(128.8e9 / 0.084 / 1e12)
    pk = bench.peaks()
    t3 = bench.gemm_roofline("lowp", "mixed_tf32x3", 1e12, 1.0, True, 0.2)
    assert t3["peak"] == pytest.approx(pk["bf16_sustained"] * bench.TF32_OVER_BF16 / 3)
    bf = bench.gemm_roofline("lowp", "mixed_bf16", 1e12, 1.0, False, 0.2)
    assert bf["peak"] == pk["bf16_burst"] and bf["bound"] == "tensor"


def test_peaks_come_from_the_measured_file_when_present():
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    pk = bench.peaks()
    if os.path.exists(path):
        d = json.load(open(path))
        assert pk["source"] == "measured" and pk["hbm_gbs"] == d["hbm_gbs"]
        assert pk["bf16_burst"] == d["bf16_tflops"] and pk["bf16_sustained"] == d["bf16_tflops_sustained"]
    else:
        assert pk == {"hbm_gbs": 6800.0, "bf16_burst": 1900.0, "bf16_sustained": 1700.0, "source": "fallback"}


def test_job_throughput_is_whole_job():
    assert bench.job_throughput(1000, 4, 2.0) == pytest.approx(1000 * 4 / 0.002)
