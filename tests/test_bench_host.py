"""Host logic of bench.py (no GPU): roofline arithmetic, measured-traffic lookup, peaks source, and the
oracle reference arm on the small dense workload."""
import json
import os
import subprocess
import sys

import pytest

import bench


def test_traffic_only_for_the_captured_workload():
    assert bench.traffic_for("k_gemm_slices<double>", "dense_n1024_s1024_p16") == 502828800 + 137370112
    assert bench.traffic_for("k_oz_sylv/6", "dense_n1024_s1024_p16") == 1566623488 + 140020736
    assert bench.traffic_for("k_gemm_slices<double>", "dense_n4096_s256_p32_g0.3") is None
    assert bench.traffic_for("k_tc_sylv", "dense_n1024_s1024_p16") is None


def test_slice_flops_counts_complex_and_real_slices():
    # n = s = 1024, p = 16: 7 complex + 2 real slices; 8 FLOP conventional, 6 for the 3-multiply form
    per = 1024 * 1024 * 2048
    assert bench.slice_flops(1024, 1024, 16, 8) == per * (8 * 7 + 2 * 2)
    assert bench.slice_flops(1024, 1024, 16, 6) == per * (6 * 7 + 2 * 2)
    assert bench.slice_flops(10, 3, 5, 8) == 10 * 3 * 13 * (8 * 2 + 2 * 1)     # odd p: no Nyquist slice
    assert bench.slice_flops(10, 3, 1, 8) == 10 * 3 * 13 * 2                   # p = 1: one real slice


def test_ozaki_roofline_counts_the_issued_digit_pairs():
    pk = bench.peaks()
    flops, ms = 128.8e9, 3.0
    r6 = bench.ozaki_roofline(flops, 21 * flops, ms, True, 0.5)
    assert r6["achieved"] == pytest.approx(21 * flops / (ms * 1e-3) / 1e12)
    assert r6["peak"] == pk["bf16_sustained"]
    assert r6["frac"] == pytest.approx(r6["achieved"] / r6["peak"])
    assert "21.0 BF16 digit-pair" in r6["kernel"]
    r = bench.ozaki_roofline(flops, (10 + 15 + 21) * flops / 3, ms, False, 0.4)
    assert r["peak"] == pk["bf16_burst"]
    assert "15.3 BF16 digit-pair" in r["kernel"]


def test_fp64_roofline_is_a_fraction_of_the_device_peak():
    """The DFMA slice GEMM executes 6 FLOPs per complex multiply-add; at the measured 84 ms per launch
    that is below the peak derived from 152 SMs at 2070 MHz, while the 8-FLOP count would exceed it."""
    ex, conv = bench.slice_flops(1024, 1024, 16, 6), bench.slice_flops(1024, 1024, 16, 8)
    r = bench.fp64_gemm_roofline(ex, conv, 84.0, 0.98, 152, 2070.0)
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(4 * 152 * 2.070e9 / 1e12)
    assert r["achieved"] == pytest.approx(ex / 0.084 / 1e12)
    assert 0.85 < r["frac"] < 1.0
    assert conv / 0.084 / 1e12 > r["peak"]
    assert bench.fp64_peak_tflops(76, 1000.0) == pytest.approx(4 * 76 * 1e9 / 1e12)


def test_lowp_roofline_peaks():
    pk = bench.peaks()
    t3 = bench.lowp_gemm_roofline("mixed_tf32x3", 1e12, 1.0, True, 0.2, 152, 2070.0)
    assert t3["peak"] == pytest.approx(pk["bf16_sustained"] * bench.TF32_OVER_BF16 / 3)
    bf = bench.lowp_gemm_roofline("mixed_bf16", 1e12, 1.0, False, 0.2, 152, 2070.0)
    assert bf["peak"] == pk["bf16_burst"] and bf["bound"] == "tensor"
    f32 = bench.lowp_gemm_roofline("mixed_fp32", 1e12, 1.0, False, 0.2, 152, 2070.0)
    assert f32["peak"] == pytest.approx(bench.ffma_peak_tflops(152, 2070.0)) and f32["bound"] == "alu"


def test_speedups_pair_every_fast_form_with_every_fp64_engine():
    e = {"fp64": {"value": 10.0}, "fp64@ozaki": {"value": 100.0}, "mixed_bf16@ozaki": {"value": 400.0},
         "mixed_tf32x3@ozaki": {"error": "x"}}
    sp = bench.speedups(e, ["fp64", "fp64@ozaki"], ["mixed_bf16@ozaki", "mixed_tf32x3@ozaki"])
    assert sp == {"mixed_bf16@ozaki / fp64": 40.0, "mixed_bf16@ozaki / fp64@ozaki": 4.0}


def test_peaks_come_from_the_measured_file_when_present():
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    pk = bench.peaks()
    if os.path.exists(path):
        d = json.load(open(path))
        assert pk["source"] == "measured" and pk["hbm_gbs"] == d["hbm_gbs"]
        assert pk["bf16_burst"] == d["bf16_tflops"] and pk["bf16_sustained"] == d["bf16_tflops_sustained"]
    else:
        assert pk["source"] == "fallback" and pk["hbm_gbs"] == 6800.0


def test_job_throughput_is_whole_job():
    assert bench.job_throughput(1000, 4, 2.0) == pytest.approx(1000 * 4 / 0.002)


def test_reference_arm_times_the_oracle_and_honours_steps():
    """The oracle arm on the small dense workload: one JSON line, the requested steps and warm-up, its
    own step time in ms_per_step, and a value in the metric's unit from a complete oracle solve."""
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "dense_n24_s24_p4", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=300, env={**os.environ, "RANK": "0"})
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["unit"] == "unknowns/s" and line["value"] > 0 and line["ms_per_step"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and "complete oracle tGMRES(20)" in line["cpu_baseline"]["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["oracle_complete_solve_s"] > 0


def test_fp64_roofline_carries_the_measured_probe():
    """The derived FP64 roof stays the denominator; the measured FMA loop is reported beside it."""
    r = bench.fp64_gemm_roofline(98.8e9, 128.8e9, 84.1, 0.97, 152, 2070.0, 1.10, 1.2554)
    assert r["peak"] == pytest.approx(4.0 * 152 * 2070e6 / 1e12)
    assert r["frac"] == pytest.approx(98.8e9 / 84.1e-3 / 1e12 / r["peak"])
    assert r["peak_probe"] == 1.2554 and "1.255 TFLOP/s" in r["note"]
    r0 = bench.fp64_gemm_roofline(98.8e9, 128.8e9, 84.1, 0.97, 152, 2070.0)
    assert r0["peak_probe"] is None and "FMA loop" not in r0["note"]


def test_fp64_probe_failure_does_not_fail_the_bench():
    class NoGpu:
        def probe_fp64_peak(self):
            raise RuntimeError("no device")

    class Fixed:
        def probe_fp64_peak(self):
            return 1.25

    assert bench.measure_fp64_probe(NoGpu()) is None
    assert bench.measure_fp64_probe(Fixed()) == 1.25
    assert bench.probe_note(None) == ""
