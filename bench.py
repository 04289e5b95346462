#!/usr/bin/env python3
"""Benchmark: Sylvester-tensor-equation unknowns solved per second, to a true relative residual
of 1e-10, on GB300.

One step = one complete solve of A*X - X*B = C from X0 = 0 through the C ABI (operator setup
ts_op_create_dense included), with the inputs resident in HBM.  The default workload is the
dense 1024 x 1024 x 16 family (A^(1) = tridiag(-1,4,-1) + 0.1 G/sqrt(n), ...; X* ~ U(-1,1),
C = M(X*)) solved by FP64 tGMRES(30) on the FP64 CUDA cores.  Every rank solves its own instance
(weak scaling, no collective on the data path).

The JSON line also carries: `e2e` (the same metric with host buffers, copies inside the timed
region, median of --e2e-steps), `roofline` for the dominant kernel (timed by CUDA events inside
the library over the timed region), `cpu_baseline` (one complete solve of the CPU oracle on this
host's cores), `clocks` sampled during the timed region, `gpu_launches`, `variants` (the other
methods, precisions and FP64 engines on the same workload, each the median of --reps timed solves
and certified by the FP64 CUDA-core operator) and `comparisons` (the mixed-precision and batched
forms against FP64 tGMRES on both FP64 engines, for the dense 1024 x 1024 x 16, the dense
4096 x 256 x 32 and the 256-instance batched workloads).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "STE unknowns/s at rel. residual 1e-10: mixed/batched vs FP64 tGMRES, 1 GB300"
UNIT = "unknowns/s"
NOMINAL_SMS = 152           # GB300, used only when no device can be queried
NOMINAL_SM_MHZ = 2070.0


def args_parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="dense_n1024_s1024_p16")
    ap.add_argument("--precision", default=None,
                    help="default: fp64 for the dense n=s=1024 workload, mixed_fp32 for the others")
    ap.add_argument("--engine", choices=["dfma", "ozaki"], default="dfma",
                    help="how FP64 applications run: FP64 CUDA cores, or emulated on the BF16 tensor cores")
    ap.add_argument("--variants", default=None,
                    help="comma list of extra precision[@engine] runs to time, 'tfom' for FP64 tFOM ('' = none; "
                         "default: every method, precision and engine the workload supports)")
    ap.add_argument("--reps", type=int, default=3, help="timed solves per variant / comparison entry (median)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparisons", action="store_true",
                    help="skip the cross-workload comparison of the mixed/batched forms with FP64 tGMRES")
    ap.add_argument("--mode", choices=["solve", "apply"], default="solve",
                    help="solve: full solves (the benchmark); apply: operator applications only (kernel runs)")
    ap.add_argument("--count", type=int, default=None, help="instances of the batched workload (default 256)")
    ap.add_argument("--n", type=int)
    ap.add_argument("--s", type=int)
    ap.add_argument("--p", type=int)
    return ap.parse_args(argv)


DENSE_VARIANTS = ("tfom,fp64+spectral,mixed_fp32,mixed_tf32x3,mixed_tf32,mixed_bf16,fp64@ozaki,fp64@ozaki+spectral,"
                  "tfom@ozaki,mixed_tf32x3@ozaki,mixed_bf16@ozaki")
BATCHED_VARIANTS = "fp64,mixed_fp32,fp64@ozaki,mixed_fp32@ozaki,mixed_tf32x3@ozaki,mixed_bf16@ozaki"
DENSE_WORKLOADS = ("dense_n24_s24_p4", "dense_n1024_s1024_p16", "dense_n4096_s256_p32_g0.3")


def workload_cfg(a):
    from paper_2405_09233_gb300 import inputs
    cfg = dict(inputs.WORKLOADS[a.workload])
    for key in ("n", "s", "p"):
        if getattr(a, key) is not None:
            cfg[key] = getattr(a, key)
    return cfg


# ------------------------------------------------------------------------------------------------
# roofline arithmetic
# ------------------------------------------------------------------------------------------------
def peaks():
    """Roofline denominators: MEASURED_PEAKS.json when present, else the recipe's fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_burst": d["bf16_tflops"], "bf16_sustained": d["bf16_tflops_sustained"],
                "sm_max_mhz": d.get("sm_max_mhz", NOMINAL_SM_MHZ), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_burst": 1900.0, "bf16_sustained": 1700.0, "sm_max_mhz": NOMINAL_SM_MHZ,
                "source": "fallback"}


def device_sms(dev=None) -> int:
    """SM count of the device (the nominal 152 when no device can be queried)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.get_device_properties(dev if dev is not None else 0).multi_processor_count)
    except Exception:
        pass
    return NOMINAL_SMS


def fp64_peak_tflops(sms: int, mhz: float) -> float:
    """FP64 CUDA-core peak derived from unit counts and clock: 2 DFMA (4 FLOP) per clock per SM."""
    return 4.0 * sms * mhz * 1e6 / 1e12


def ffma_peak_tflops(sms: int, mhz: float) -> float:
    """FP32 CUDA-core peak: 128 FP32 lanes per SM, 2 FLOP per FMA."""
    return 2.0 * 128 * sms * mhz * 1e6 / 1e12


TF32_OVER_BF16 = 1.1 / 2.25       # nominal dense tensor rates (PFLOP/s per GPU)


def slice_flops(n, s, p, per_complex):
    """FLOPs of one application's slice products Y_k = A_k X_k - X_k B_k over the K = p/2 + 1 Fourier
    slices, at `per_complex` FLOPs per complex multiply-add (8 conventional, 6 for the three-multiply
    form) and 2 per real one (slices 0 and p/2)."""
    K = p // 2 + 1
    nreal = 1 + (1 if p % 2 == 0 and p > 1 else 0)
    return n * s * (n + s) * (per_complex * (K - nreal) + 2 * nreal)


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the dominant kernels at the
# n = s = 1024, p = 16 workload, from one ncu capture each of the kernels as they stand; a roofline object
# carries them only for that workload and, for the emulated product, only when every launch used 6 digits.
TRAFFIC_N1024 = {"k_gemm_slices<double>": 502828800 + 137370112, "k_oz_sylv/6": 1566623488 + 140020736}


def traffic_for(kernel, workload):
    return TRAFFIC_N1024.get(kernel) if workload == "dense_n1024_s1024_p16" else None


def ozaki_roofline(flops_per_launch, pair_flops_per_launch, avg_ms, sustained, share):
    """Emulated FP64 slice products: the tensor pipe executes S(S+1)/2 BF16 digit-pair products per
    algorithmic FP64 product (S per launch: 6, or fewer for the early residuals of a mixed solve);
    achieved = those BF16 FLOPs / launch time (digit split included)."""
    pk = peaks()
    peak = pk["bf16_sustained"] if sustained else pk["bf16_burst"]
    pairs = pair_flops_per_launch / max(flops_per_launch, 1e-30)
    achieved = pair_flops_per_launch / (avg_ms * 1e-3) / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "kernel": "k_oz_sylv (emulated FP64: %.1f BF16 digit-pair products per launch on tcgen05)" % pairs,
            "note": "peak: %s BF16 %s (of measured); FP64-equivalent rate %.2f TFLOP/s (8 FLOP per complex "
                    "multiply-add). Kernel share of the step: %.3f"
                    % (pk["source"], "sustained" if sustained else "burst",
                       flops_per_launch / (avg_ms * 1e-3) / 1e12, share)}


def fp64_gemm_roofline(executed_per_launch, conventional_per_launch, avg_ms, share, sms, mhz, dgemm_tflops=None,
                       probe_tflops=None):
    """The FP64 CUDA-core slice GEMM.  It implements the three-multiplication (Gauss) complex product,
    whose FLOP count is 6 per complex multiply-add (3 DFMA) and 2 per real one: achieved = that count
    / launch time, against the FP64 peak derived from the device's SM count and maximum clock."""
    peak = fp64_peak_tflops(sms, mhz)
    achieved = executed_per_launch / (avg_ms * 1e-3) / 1e12
    conv = conventional_per_launch / (avg_ms * 1e-3) / 1e12
    note = (f"FLOPs of the 3-multiply complex product the kernel implements (6 per complex multiply-add, 2 per "
            f"real); the conventional 8-FLOP count gives {conv:.3f} TFLOP/s. peak derived: 2 DFMA/clk/SM x "
            f"{sms} SMs x {mhz:.0f} MHz. Kernel share of the step: {share:.3f}")
    if dgemm_tflops:
        note += f". cuBLAS DGEMM (8192^3, torch) in this run: {dgemm_tflops:.3f} TFLOP/s"
    note += probe_note(probe_tflops)
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": "k_gemm_slices<double> (FP64 DFMA, 3-multiply complex)", "note": note,
            "peak_probe": probe_tflops}


def probe_note(probe_tflops):
    return (f". Measured FP64 FMA loop (ts_probe_fp64_peak, 8 independent chains per thread) in this run: "
            f"{probe_tflops:.3f} TFLOP/s" if probe_tflops else "")


def measure_fp64_probe(ctx):
    """The FP64 roof measured on the device by the library's FMA loop (a cross-check of the derived one)."""
    try:
        return ctx.probe_fp64_peak()
    except Exception:   # report the run without it rather than fail the bench
        return None


def lowp_gemm_roofline(precision, flops_per_launch, avg_ms, sustained, share, sms, mhz):
    """The low-precision slice products: FP32 CUDA cores, or tcgen05 with TF32 / BF16 / split-TF32 inputs."""
    achieved = flops_per_launch / (avg_ms / 1e3) / 1e12
    pk = peaks()
    if precision == "mixed_fp32":
        peak = ffma_peak_tflops(sms, mhz)
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "k_gemm_slices<float> (FP32 FFMA)",
                "note": f"peak derived: 2 FLOP x 128 lanes/SM x {sms} SMs x {mhz:.0f} MHz. Kernel share: {share:.3f}"}
    bf = pk["bf16_sustained"] if sustained else pk["bf16_burst"]
    tf32 = precision in ("mixed_tf32", "mixed_tf32x3")
    parts = 3 if precision == "mixed_tf32x3" else 1
    peak = bf * (TF32_OVER_BF16 if tf32 else 1.0) / parts
    name = {"mixed_tf32": "TF32", "mixed_bf16": "BF16", "mixed_tf32x3": "split TF32 x3"}[precision]
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": f"k_tc_sylv ({name} tcgen05)",
            "note": (f"peak: {pk['source']} BF16 {'sustained' if sustained else 'burst'} (of measured)"
                     + (" x nominal TF32/BF16 ratio 0.489" if tf32 else "")
                     + (" / 3 products (split TF32)" if parts == 3 else "")
                     + f"; 8 FLOP per complex multiply-add. Kernel share of the step: {share:.3f}")}


def stats_rooflines(st, n, s, p, total_ms, sustained, precision, sms, mhz, workload, dgemm=None, exec_ratio=None,
                    probe=None):
    """Roofline objects of every slice-product class the library timed; the first is the dominant one.
    exec_ratio (batched workloads): executed / conventional FLOPs of the FP64 products over the batch."""
    out = []
    batched = exec_ratio is not None
    if st.gemm_launches:
        if batched:
            conv = st.gemm_flops / st.gemm_launches
            executed = conv * exec_ratio
        else:
            conv, executed = slice_flops(n, s, p, 8), slice_flops(n, s, p, 6)
        r = fp64_gemm_roofline(executed, conv, st.gemm_ms / st.gemm_launches, st.gemm_ms / total_ms, sms, mhz, dgemm,
                               probe)
        if not batched:
            r["traffic"] = traffic_for("k_gemm_slices<double>", workload)
        out.append((st.gemm_ms, r))
    if st.oz_launches:
        r = ozaki_roofline(st.oz_flops / st.oz_launches, st.oz_pair_flops / st.oz_launches,
                           st.oz_ms / st.oz_launches, sustained, st.oz_ms / total_ms)
        if not batched and abs(st.oz_pair_flops - 21 * st.oz_flops) <= 1e-9 * st.oz_pair_flops:
            r["traffic"] = traffic_for("k_oz_sylv/6", workload)
        out.append((st.oz_ms, r))
    if st.lowp_launches and precision != "fp64":
        r = lowp_gemm_roofline(precision, st.lowp_flops / st.lowp_launches, st.lowp_ms / st.lowp_launches,
                               sustained, st.lowp_ms / total_ms, sms, mhz)
        out.append((st.lowp_ms, r))
    out.sort(key=lambda t: -t[0])
    return [r for _, r in out]


def max_over_ranks(value: float, device=None) -> float:
    """The slowest rank's time: all-reduce MAX over the process group (NCCL on GPUs, gloo on CPU)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job throughput: every rank processed its own units, the job took the slowest rank's time."""
    return units_per_rank * world / (ms_max / 1e3)


def rank_seed(rank: int) -> int:
    """Each rank solves its own instance of the workload family (weak scaling)."""
    return 1 + rank


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def blas_threads():
    """Threads numpy's BLAS uses (threadpoolctl when importable, else the host's core count)."""
    try:
        from threadpoolctl import threadpool_info
        n = [d.get("num_threads") for d in threadpool_info() if d.get("user_api") == "blas"]
        if n and n[0]:
            return int(n[0])
    except Exception:
        pass
    return os.cpu_count()


def speedups(entries, base_names, fast_names):
    """value(fast) / value(base) for every pair present without error."""
    out = {}
    for f in fast_names:
        for b in base_names:
            if f in entries and b in entries and "value" in entries[f] and "value" in entries[b]:
                out[f"{f} / {b}"] = entries[f]["value"] / entries[b]["value"]
    return out


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": statistics.median(power) if power else None}


def measure_dgemm_tflops(dev):
    """cuBLAS FP64 GEMM rate (torch.matmul, 8192^3, best of 3): a measured reference for the FP64 roof."""
    try:
        import torch
        a = torch.randn(8192, 8192, dtype=torch.float64, device=dev)
        b = torch.randn(8192, 8192, dtype=torch.float64, device=dev)
        torch.matmul(a, b)
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        del a, b
        torch.cuda.empty_cache()
        return 2 * 8192 ** 3 / (best * 1e-3) / 1e12
    except Exception:
        return None


# ------------------------------------------------------------------------------------------------
# the CPU oracle (rank 0, N = 1)
# ------------------------------------------------------------------------------------------------
def oracle_dense_inputs(wl_cfg, seed):
    """The workload's inputs with C = M(X*) formed by the oracle (never by the CUDA path)."""
    from paper_2405_09233_gb300 import inputs
    from oracle import krylov
    pr = inputs.dense_problem(wl_cfg["n"], wl_cfg["s"], wl_cfg["p"], seed=seed, scale=wl_cfg["scale"])
    return pr, krylov.sylv_apply(pr.A, pr.B, pr.Xstar)


def oracle_full_solve(pr, C, restart):
    """One complete oracle tGMRES(m) solve (Algorithm 3 over the bcirc definition), timed."""
    from oracle import krylov
    t0 = time.perf_counter()
    r = krylov.tgmres(pr.A, pr.B, C, m=restart, tol=1e-10)
    return time.perf_counter() - t0, r


def cpu_baseline_dense(wl_cfg, seed):
    n, s, p = wl_cfg["n"], wl_cfg["s"], wl_cfg["p"]
    pr, C = oracle_dense_inputs(wl_cfg, seed)
    t, r = oracle_full_solve(pr, C, wl_cfg["restart"])
    return {"value": n * s * p / t, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
            "sample": (f"one complete oracle tGMRES({wl_cfg['restart']}) solve at n={n}, s={s}, p={p} (timed solve, "
                       f"MGS included; numpy FP64, T-product by the bcirc block-row definition): {t:.1f} s, "
                       f"{r.iters} inner steps in {r.cycles} cycles, status {r.status}, true rel. residual "
                       f"{r.relres:.2e}")}


def cpu_baseline_batched(specs, budget_s=20.0):
    """Complete oracle tGMRES(20) solves of the batch's instances in their order, until ~budget_s."""
    from paper_2405_09233_gb300 import inputs
    from oracle import krylov
    solved, t_tot, unknowns = 0, 0.0, 0
    for sp in specs:
        pr = inputs.dense_problem(sp.n, sp.s, sp.p, seed=sp.seed)
        C = krylov.sylv_apply(pr.A, pr.B, pr.Xstar)
        t0 = time.perf_counter()
        krylov.tgmres(pr.A, pr.B, C, m=20, tol=1e-10)
        t_tot += time.perf_counter() - t0
        unknowns += sp.n * sp.s * sp.p
        solved += 1
        if t_tot >= budget_s:
            break
    return {"value": unknowns / t_tot, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
            "sample": (f"complete oracle tGMRES(20) solves (FP64, bcirc definition) of the batch's first {solved} "
                       f"instances in their order ({unknowns} unknowns, {t_tot:.1f} s)")}


def cpu_baseline_tbas(prob, m):
    import scipy.sparse as sp
    from oracle import tubal
    slices = [sp.csr_matrix((sl.val, sl.col, sl.rowptr), shape=(prob.n, prob.n)) for sl in prob.slices]
    applyA = lambda Z: tubal.tprod_sparse(slices, Z)  # noqa: E731
    from oracle import tproduct
    C = applyA(prob.Xstar) - tproduct.tprod(prob.Xstar, prob.B)
    t0 = time.perf_counter()
    r = tubal.tbas(None, prob.B, C, m=m, tol=1e-10, applyA=applyA)
    t = time.perf_counter() - t0
    return {"value": prob.n * prob.B.shape[0] * prob.p / t, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
            "sample": (f"one complete oracle TBAS({m}) solve at n={prob.n}, s={prob.B.shape[0]}, p={prob.p} (timed "
                       f"solve; sparse frontal slices, bcirc block-row T-products): {t:.1f} s, {r.cycles} cycles, "
                       f"status {r.status}")}


def run_reference(a):
    """The reference arm: the oracle on this host's cores, on the default workload's config.

    A complete oracle tGMRES(30) solve is timed once first (calibration).  Each warm-up and timed step
    is then a bounded sample of the same solve: one inner step of the oracle's Algorithm 2 at the full
    size (one M(X) by the bcirc definition, the MGS pass, the norm), about 1/S of the complete solve's
    time, S = T(complete solve) / T(sample) from the calibration.  ms_per_step is the sample's own
    time; value = unknowns / (median step x S)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    from paper_2405_09233_gb300 import inputs
    from oracle import krylov
    if a.workload not in ("dense_n1024_s1024_p16", "dense_n24_s24_p4"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the dense workloads only"}))
        return
    cfg = inputs.WORKLOADS[a.workload]
    n, s, p, m = cfg["n"], cfg["s"], cfg["p"], cfg["restart"]
    pr, C = oracle_dense_inputs(cfg, 1)
    apply = lambda X: krylov.sylv_apply(pr.A, pr.B, X)  # noqa: E731
    V = C / np.linalg.norm(C)

    def sample():
        t0 = time.perf_counter()
        krylov.tarnoldi(apply, V, 1)
        return time.perf_counter() - t0

    t_full, r = oracle_full_solve(pr, C, m)
    t_cal = sample()
    S = t_full / t_cal
    for _ in range(a.warmup):
        sample()
    ts = [sample() for _ in range(a.steps)]
    t_step = statistics.median(ts)
    value = n * s * p / (t_step * S)
    cores = blas_threads()
    desc = (f"calibration: one complete oracle tGMRES({m}) solve ({t_full:.1f} s, {r.iters} inner steps, "
            f"{r.cycles} cycles, status {r.status}) = {S:.1f} samples of {t_cal:.2f} s; each step = one inner step "
            f"of the oracle's Algorithm 2 at full size (M(X) by the bcirc definition, MGS pass, norm); "
            f"value = unknowns / (median step x {S:.1f})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * statistics.mean(ts),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": a.workload, "n": n, "s": s, "p": p, "restart": m, "tol": 1e-10},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "oracle_complete_solve_s": t_full}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
# dense and batched measurement helpers
# ------------------------------------------------------------------------------------------------
class DenseSetup:
    """Device-resident inputs of one dense workload instance; C = M(X*) by the library's FP64 operator."""

    def __init__(self, ctx, wl, seed, dev, n=None, s=None, p=None, pinned=False):
        import torch
        from paper_2405_09233_gb300 import inputs
        cfg = dict(inputs.WORKLOADS[wl])
        for key, v in (("n", n), ("s", s), ("p", p)):
            if v is not None:
                cfg[key] = v
        self.cfg, self.wl = cfg, wl
        self.n, self.s, self.p, self.m = cfg["n"], cfg["s"], cfg["p"], cfg["restart"]
        pr = inputs.dense_problem(self.n, self.s, self.p, seed=seed, scale=cfg["scale"])
        A_h = torch.from_numpy(inputs.to_device_layout(pr.A))
        B_h = torch.from_numpy(inputs.to_device_layout(pr.B))
        Xs_h = torch.from_numpy(inputs.to_device_layout(pr.Xstar))
        if pinned:
            A_h, B_h, Xs_h = A_h.pin_memory(), B_h.pin_memory(), Xs_h.pin_memory()
        self.A_h, self.B_h = A_h, B_h
        self.Ad, self.Bd, self.Xs = A_h.to(dev), B_h.to(dev), Xs_h.to(dev)
        del pr
        self.ctx = ctx
        self.op_cert = ctx.op_create_dense(self.Ad, self.Bd)     # the FP64 CUDA-core operator (certificates)
        self.Cd = ctx.sylv_apply(self.op_cert, self.Xs)
        self.normC = float(torch.linalg.norm(self.Cd))
        self.X = torch.zeros_like(self.Cd)
        self.unknowns = self.n * self.s * self.p
        torch.cuda.synchronize()

    def solve(self, name):
        """One step: operator setup + solve from X0 = 0.  name = method-or-precision[@engine][+spectral]:
        "tfom" = FP64 tFOM, else a tGMRES precision; "+spectral" keeps the FP64 Krylov basis in the
        Fourier domain."""
        base, _, flag = name.partition("+")
        prec, _, eng = base.partition("@")
        eng = eng or "dfma"
        spectral = flag == "spectral"
        op = self.ctx.op_create_dense(self.Ad, self.Bd)
        self.X.zero_()
        if prec == "tfom":
            r = self.ctx.tfom_solve(op, self.Cd, self.X, restart=self.m, tol=1e-10, engine=eng, spectral=spectral)
        else:
            r = self.ctx.tgmres_solve(op, self.Cd, self.X, restart=self.m, tol=1e-10, precision=prec, engine=eng,
                                      spectral=spectral)
        op.close()
        return r

    def certify(self):
        """||C - M(X)|| / ||C|| with the FP64 CUDA-core operator (outside any timed region)."""
        import torch
        R = self.Cd - self.ctx.sylv_apply(self.op_cert, self.X)
        return float(torch.linalg.norm(R)) / self.normC

    def err_xstar(self):
        import torch
        return float(torch.max(torch.abs(self.X - self.Xs)) / torch.max(torch.abs(self.Xs)))

    def close(self):
        self.op_cert.close()


def timed_median(fn, reps, warm):
    """warm untimed calls, then reps calls each timed with CUDA events; returns (median ms, list, last result)."""
    import torch
    r = None
    for _ in range(warm):
        r = fn()
    ms = []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms), ms, r


def dense_entry(setup, name, reps, warm=1, world=1):
    """Median of reps timed solves of one method / precision / engine, with its FP64 certificate."""
    try:
        med, ms, r = timed_median(lambda: setup.solve(name), reps, warm)
        return {"value": setup.unknowns * world / (med / 1e3), "ms_per_step": med, "ms_all": ms,
                "status": r.status_name, "relres_true": r.info.relres_true, "relres_fp64_dfma": setup.certify(),
                "outer": r.info.outer, "inner_iters": r.info.iters, "applies_fp64": r.info.applies_fp64,
                "applies_low": r.info.applies_low, "err_vs_xstar": setup.err_xstar()}
    except Exception as e:  # report, do not hide
        return {"error": str(e)}


class BatchedSetup:
    """The batched workload: `count` dense-family instances (n log-uniform in [64, 1024], s uniform in
    [16, 128], p in {4, 8, 16}), device-resident; C_i = M_i(X*_i) by the library's FP64 operator."""

    def __init__(self, ctx, count, seed, dev, pinned=False):
        import torch
        from paper_2405_09233_gb300 import inputs
        self.ctx, self.count = ctx, count
        self.specs = inputs.batched_specs(count, seed=seed)
        self.host = []
        for sp in self.specs:
            pr = inputs.dense_problem(sp.n, sp.s, sp.p, seed=sp.seed)
            t = (torch.from_numpy(inputs.to_device_layout(pr.A)), torch.from_numpy(inputs.to_device_layout(pr.B)),
                 torch.from_numpy(inputs.to_device_layout(pr.Xstar)))
            self.host.append(tuple(x.pin_memory() for x in t) if pinned else t)
        self.dev_in = [(A.to(dev), B.to(dev), X.to(dev)) for A, B, X in self.host]
        self.ops_cert = [ctx.op_create_dense(A, B) for A, B, _ in self.dev_in]
        self.Cs = [ctx.sylv_apply(op, Xst) for op, (_, _, Xst) in zip(self.ops_cert, self.dev_in)]
        self.normC = [float(torch.linalg.norm(C)) for C in self.Cs]
        self.Xs = [torch.zeros_like(C) for C in self.Cs]
        self.unknowns = sum(sp.n * sp.s * sp.p for sp in self.specs)
        torch.cuda.synchronize()

    def solve(self, name):
        """One step: create the batch's operators, solve them together, release the operators.  The host
        time of each part of the last call is kept in self.split_ms."""
        import torch
        prec, _, eng = name.partition("@")
        t0 = time.perf_counter()
        ops = [self.ctx.op_create_dense(A, B) for A, B, _ in self.dev_in]
        for X in self.Xs:
            X.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        st, infos, _ = self.ctx.batched_solve(ops, self.Cs, self.Xs, restart=20, tol=1e-10, precision=prec,
                                              engine=eng or "dfma")
        t2 = time.perf_counter()
        for op in ops:
            op.close()
        t3 = time.perf_counter()
        self.split_ms = {"op_create": 1e3 * (t1 - t0), "solve": 1e3 * (t2 - t1), "op_destroy": 1e3 * (t3 - t2),
                         "solve_device_ms": infos[0].ms_total if infos else None}
        return st, infos

    def certify(self):
        import torch
        return max(float(torch.linalg.norm(C - self.ctx.sylv_apply(op, X))) / nc
                   for op, C, X, nc in zip(self.ops_cert, self.Cs, self.Xs, self.normC))

    def err_xstar(self):
        import torch
        return max(float(torch.max(torch.abs(X - Xst))) for X, (_, _, Xst) in zip(self.Xs, self.dev_in))

    def close(self):
        for op in self.ops_cert:
            op.close()


def batched_entry(setup, name, reps, warm=1, world=1):
    try:
        med, ms, (st, infos) = timed_median(lambda: setup.solve(name), reps, warm)
        return {"value": setup.unknowns * world / (med / 1e3), "ms_per_step": med, "ms_all": ms, "status": st,
                "max_relres_true": max(i.relres_true for i in infos), "max_relres_fp64_dfma": setup.certify(),
                "max_err_vs_xstar": setup.err_xstar(), "max_outer": max(i.outer for i in infos),
                "split_ms_last": setup.split_ms}
    except Exception as e:  # report, do not hide
        return {"error": str(e)}


def run_comparisons(ctx, dev, reps, dense1=None, dense1_entries=None):
    """The metric's comparison: the mixed-precision and batched forms against FP64 tGMRES on both FP64
    engines (CUDA cores and the emulated tensor-core product), each entry the median of `reps` timed solves
    and certified by the FP64 CUDA-core operator."""
    import torch
    out = {}
    fp64s = ["fp64", "fp64@ozaki", "fp64@ozaki+spectral"]
    fast = ["mixed_bf16@ozaki", "mixed_tf32x3@ozaki"]
    if dense1 is not None and dense1_entries is not None:
        out["dense_n1024_s1024_p16"] = {"entries": dense1_entries,
                                        "speedup": speedups(dense1_entries, fp64s, fast)}
    try:
        d2 = DenseSetup(ctx, "dense_n4096_s256_p32_g0.3", 1, dev)
        ent = {"fp64": dense_entry(d2, "fp64", 1, warm=0)}
        for nm in ("fp64@ozaki", "fp64@ozaki+spectral", "mixed_tf32x3@ozaki", "mixed_bf16@ozaki"):
            ent[nm] = dense_entry(d2, nm, reps)
        out["dense_n4096_s256_p32_g0.3"] = {"entries": ent, "speedup": speedups(ent, fp64s, fast)}
        d2.close()
        del d2
        torch.cuda.empty_cache()
    except Exception as e:  # report, do not hide
        out["dense_n4096_s256_p32_g0.3"] = {"error": str(e)}
    try:
        b = BatchedSetup(ctx, 256, 4, dev)
        ent = {nm: batched_entry(b, nm, reps) for nm in ("fp64", "fp64@ozaki", "mixed_bf16@ozaki",
                                                          "mixed_tf32x3@ozaki")}
        out["batched_256"] = {"entries": ent, "speedup": speedups(ent, fp64s, fast)}
        b.close()
        del b
        torch.cuda.empty_cache()
    except Exception as e:  # report, do not hide
        out["batched_256"] = {"error": str(e)}
    return out


# ------------------------------------------------------------------------------------------------
def main():
    a = args_parse()
    if a.variants is None:
        a.variants = BATCHED_VARIANTS if a.workload == "batched_256" else DENSE_VARIANTS
    if a.precision is None:
        a.precision = ("fp64" if a.workload in ("dense_n24_s24_p4", "dense_n1024_s1024_p16", "sparse_lap128_s32_p8")
                       else "mixed_fp32")
    if a.impl == "reference":
        run_reference(a)
        return
    import torch
    from paper_2405_09233_gb300 import Context

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if a.workload in ("batched_256", "sparse_lap128_s32_p8"):
        (run_batched if a.workload == "batched_256" else run_tbas)(a, rank, world, local, dev)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    ctx = Context(local)
    if a.mode == "apply":
        cfg = workload_cfg(a)
        su = DenseSetup(ctx, a.workload, rank_seed(rank), dev, a.n, a.s, a.p)
        su.close()
        return run_apply_mode(a, ctx, su.Ad, su.Bd, su.Xs, cfg, world, dev)
    su = DenseSetup(ctx, a.workload, rank_seed(rank), dev, a.n, a.s, a.p, pinned=True)
    n, s, p, m = su.n, su.s, su.p, su.m
    primary = a.precision + ("" if a.engine == "dfma" else "@" + a.engine)

    for _ in range(a.warmup):
        r = su.solve(primary)
        assert r.status == 0, r

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # Small problems run their restart cycles as CUDA graphs, which per-kernel event timing would turn
    # off: they are timed with statistics off, and the kernel split comes from one extra solve.
    small = su.unknowns <= 1 << 20
    ctx.stats_reset()
    ctx.stats_enable(not small)
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    ev0.record()
    results = [su.solve(primary) for _ in range(a.steps)]
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ctx.stats_enable(False)
    st = ctx.stats_get()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / a.steps, dev)
    launches = int(st.launches)
    host_split = {"graph_build_ms_per_step": st.graph_build_ms / a.steps}
    kernel_steps, kernel_ms = a.steps, ms * a.steps
    if small:
        ctx.stats_reset()
        ctx.stats_enable(True)
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0.record()
        su.solve(primary)
        k1.record()
        torch.cuda.synchronize()
        ctx.stats_enable(False)
        st = ctx.stats_get()
        kernel_steps, kernel_ms = 1, k0.elapsed_time(k1)
    last = results[-1]
    assert all(r.status == 0 for r in results), results
    relres_cert = su.certify()
    err_xstar = su.err_xstar()
    value = job_throughput(su.unknowns, world, ms)

    sms = device_sms(dev)
    mhz = clk.get("sm_max_mhz") or peaks()["sm_max_mhz"]
    dgemm = measure_dgemm_tflops(dev) if rank == 0 and st.gemm_launches else None
    probe = measure_fp64_probe(ctx) if rank == 0 and st.gemm_launches else None
    rooflines = stats_rooflines(st, n, s, p, kernel_ms, True, a.precision, sms, mhz, a.workload, dgemm,
                                probe=probe)
    if small:
        for r in rooflines:
            r["note"] += ("; latency-bound workload: a roofline fraction says little here (the kernel split is "
                          "from one extra solve with per-kernel event timing, which runs the cycle step by step)")
    roofline = rooflines[0] if rooflines else None
    kernel_times = {"fp64_gemm_ms": st.gemm_ms / kernel_steps, "ozaki_gemm_ms": st.oz_ms / kernel_steps,
                    "lowp_gemm_ms": st.lowp_ms / kernel_steps,
                    "fft_ms": st.fft_ms / kernel_steps, "fp64_gemm_launches": st.gemm_launches // kernel_steps,
                    "ozaki_gemm_launches": st.oz_launches // kernel_steps,
                    "lowp_gemm_launches": st.lowp_launches // kernel_steps,
                    "fft_gbs": st.fft_bytes / max(st.fft_ms, 1e-9) / 1e6, "from_steps": kernel_steps}

    # end to end through the C ABI with host buffers (copies inside the timed region)
    C_h = su.Cd.cpu().pin_memory()
    X_h = torch.zeros_like(C_h).pin_memory()
    e2e_times, e2e_parts = [], []
    for _ in range(max(a.e2e_steps, 0)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op = ctx.op_create_dense(su.A_h, su.B_h)
        t1 = time.perf_counter()
        X_h.zero_()
        r = ctx.tgmres_solve(op, C_h, X_h, restart=m, tol=1e-10, precision=a.precision, engine=a.engine)
        t2 = time.perf_counter()
        op.close()
        t3 = time.perf_counter()
        e2e_times.append(t3 - t0)
        e2e_parts.append((t1 - t0, t2 - t1, t3 - t2))
        assert r.status == 0, r
    e2e = {"value": su.unknowns * world / statistics.median(e2e_times) if e2e_times else None, "unit": UNIT,
           "h2d_bytes_per_step": 8 * (n * n * p + s * s * p + 2 * n * s * p),
           "d2h_bytes_per_step": 8 * n * s * p, "steps": len(e2e_times), "statistic": "median"}
    if e2e_parts:   # host-clock split of the median end-to-end step: operator setup, solve, release
        mid = sorted(range(len(e2e_times)), key=lambda i: e2e_times[i])[len(e2e_times) // 2]
        e2e["split_ms"] = dict(zip(("op_create", "solve", "op_destroy"), (round(x * 1e3, 3) for x in e2e_parts[mid])))

    variants = {}
    for name in [v for v in a.variants.split(",") if v and v != primary]:
        variants[name] = dense_entry(su, name, a.reps, warm=1, world=world)

    if su.unknowns <= 1 << 16:
        # Small problems are latency bound.  The default path launches a cycle's steps ahead behind a
        # device gate (no host round trip per step); also time the same solve with one host round trip
        # per step, and the batched solver on this single instance (one CUDA graph per restart cycle).
        variants["us_per_inner_step"] = 1e3 * ms / max(last.info.iters, 1)
        try:
            os.environ["TSTAR_NO_LAUNCH_AHEAD"] = "1"
            med, _, r1 = timed_median(lambda: su.solve(a.precision), 20, 3)
            variants["host_round_trip_per_step"] = {
                "ms_per_step": med, "status": r1.status, "inner_iters": r1.info.iters,
                "us_per_inner_step": 1e3 * med / max(r1.info.iters, 1)}
        except Exception as e:  # report, do not hide
            variants["host_round_trip_per_step"] = {"error": str(e)}
        finally:
            os.environ.pop("TSTAR_NO_LAUNCH_AHEAD", None)
        try:
            ops1 = [ctx.op_create_dense(su.Ad, su.Bd)]

            def one():
                su.X.zero_()
                return ctx.batched_solve(ops1, [su.Cd], [su.X], restart=m, tol=1e-10, precision=a.precision)
            med, _, (stb, infb, _) = timed_median(one, 20, 3)
            variants["batched_solver_one_instance"] = {
                "value": su.unknowns * world / (med / 1e3), "ms_per_step": med, "status": stb,
                "inner_iters": infb[0].iters, "relres_true": infb[0].relres_true,
                "us_per_inner_step": 1e3 * med / max(infb[0].iters, 1)}
            ops1[0].close()
        except Exception as e:  # report, do not hide
            variants["batched_solver_one_instance"] = {"error": str(e)}

    comparisons = None
    if rank == 0 and world == 1 and not a.no_comparisons and a.workload == "dense_n1024_s1024_p16":
        d1 = {primary: {"value": value, "ms_per_step": ms, "relres_fp64_dfma": relres_cert, "status": "ok"}}
        for nm in ("fp64@ozaki", "fp64@ozaki+spectral", "mixed_bf16@ozaki", "mixed_tf32x3@ozaki"):
            if nm in variants:
                d1[nm] = variants[nm]
        comparisons = run_comparisons(ctx, dev, a.reps, su, d1)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline and a.workload in ("dense_n1024_s1024_p16",
                                                                                "dense_n24_s24_p4"):
        cpu = cpu_baseline_dense(su.cfg, rank_seed(rank))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if a.precision == "fp64" else "f32+f64",
                "data": "synthetic",
                "config": {"workload": a.workload, "n": n, "s": s, "p": p, "restart": m, "tol": 1e-10,
                           "precision": a.precision, "fp64_engine": a.engine, "method": "tGMRES",
                           "l2": "inputs larger than L2 "
                           "(A-hat 151 MB, Krylov basis 4.2 GB at n=s=1024, p=16)",
                           "iters": last.info.iters, "cycles": last.info.cycles,
                           "applies_fp64": last.info.applies_fp64, "relres_true": last.info.relres_true,
                           "relres_fp64_dfma": relres_cert, "err_vs_xstar": err_xstar, "sms": sms},
                "e2e": e2e, "roofline": roofline, "rooflines": rooflines, "cpu_baseline": cpu, "clocks": clk,
                "gpu_launches": launches, "kernels_per_step": kernel_times, "host_split": host_split,
                "variants": variants, "comparisons": comparisons}
        print(json.dumps(line), flush=True)
    su.close()
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batched(a, rank, world, local, dev):
    """The batched workload: 256 instances (n log-uniform in [64, 1024], s uniform in [16, 128],
    p in {4, 8, 16}), one step = one ts_batched_solve of all of them (operator setup included)."""
    import torch
    from paper_2405_09233_gb300 import Context
    count = a.count if a.count else 256
    ctx = Context(local)
    b = BatchedSetup(ctx, count, 4 + rank, dev, pinned=True)
    prec = a.precision
    primary = prec + ("" if a.engine == "dfma" else "@" + a.engine)
    for _ in range(a.warmup):
        st, infos = b.solve(primary)
        assert st == 0, st
    # Timed with statistics off: per-phase event timing needs the flat cycle graph, while the timed
    # steps run the nested one (a cycle stops as soon as no instance iterates).  The phase split
    # comes from one extra instrumented step.
    ctx.stats_reset()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.steps):
        st, infos = b.solve(primary)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    sth = ctx.stats_get()                       # host phases and launches of the timed steps
    step_split = dict(b.split_ms)
    ms = max_over_ranks(e0.elapsed_time(e1) / a.steps, dev)
    ctx.stats_reset()
    ctx.stats_enable(True)
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record()
    b.solve(primary)
    k1.record()
    torch.cuda.synchronize()
    ctx.stats_enable(False)
    stt = ctx.stats_get()
    instrumented_ms = k0.elapsed_time(k1)
    assert st == 0, st
    relres = max(i.relres_true for i in infos)
    cert = b.certify()
    err = b.err_xstar()
    sms = device_sms(dev)
    mhz = clk.get("sm_max_mhz") or peaks()["sm_max_mhz"]
    ratio = (sum(slice_flops(sp.n, sp.s, sp.p, 6) for sp in b.specs)
             / sum(slice_flops(sp.n, sp.s, sp.p, 8) for sp in b.specs))
    rooflines = stats_rooflines(stt, 0, 0, 0, instrumented_ms, True, prec, sms, mhz, "batched_256", exec_ratio=ratio)
    for r in rooflines:
        r["note"] += ("; batched: from one extra step whose flat cycle graph times every product phase with events "
                      "recorded in the graph, its work counted for the instances active in that phase (masked "
                      "instances' CTAs exit early and still count in the time); that step took %.1f ms"
                      % instrumented_ms)
    # end to end: operators and right-hand sides from pinned host memory, solutions back to host
    C_h = [C.cpu().pin_memory() for C in b.Cs]
    X_h = [torch.zeros_like(C).pin_memory() for C in C_h]
    t_e2e = []
    for _ in range(max(a.e2e_steps, 1)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ops = [ctx.op_create_dense(A, B) for A, B, _ in b.host]
        Cd = [C.to(dev, non_blocking=True) for C in C_h]
        Xd = [torch.zeros_like(C) for C in Cd]
        st2, _, _ = ctx.batched_solve(ops, Cd, Xd, restart=20, tol=1e-10, precision=prec, engine=a.engine)
        for Xh_, Xd_ in zip(X_h, Xd):
            Xh_.copy_(Xd_, non_blocking=True)
        torch.cuda.synchronize()
        t_e2e.append(time.perf_counter() - t0)
        for op in ops:
            op.close()
        assert st2 == 0, st2
    h2d = sum(8 * (A.numel() + B.numel() + C.numel()) for (A, B, _), C in zip(b.host, C_h))
    d2h = sum(8 * X.numel() for X in X_h)
    variants = {}
    for name in [v for v in (a.variants or "").split(",") if v and v != primary]:
        variants[name] = batched_entry(b, name, a.reps, warm=1, world=world)
    cpu = cpu_baseline_batched(b.specs) if rank == 0 and world == 1 and not a.no_cpu_baseline else None
    # the autotuner's choice for the batched tensor-core products: column tile, and whether the
    # persistent kernel (one CTA per SM walking the work list) won over one CTA per work item
    tc_schedule, simt_tiles = None, {}
    for key_, v in ctx.tune_entries().items():
        if key_.startswith("btc:"):
            tc_schedule = {"column_tile": v & ~1, "persistent": bool(v & 1)}
        elif key_.startswith("bsimt:"):     # CUDA-core products' column width, per element size
            simt_tiles["fp64" if key_.startswith("bsimt:8:") else "fp32"] = v
    if rank == 0:
        line = {"metric": METRIC, "value": b.unknowns * world / (ms / 1e3), "unit": UNIT, "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64" if prec != "fp64" else "f64", "data": "synthetic",
                "config": {"workload": "batched_256" if count == 256 else "batched_%d" % count, "instances": count,
                           "unknowns": b.unknowns, "restart": 20,
                           "tol": 1e-10, "precision": prec, "fp64_engine": a.engine, "method": "batched tGMRES",
                           "max_relres_true": relres, "max_relres_fp64_dfma": cert, "max_err_vs_xstar": err,
                           "l2": "inputs larger than L2 (5 GB basis)", "sms": sms,
                           "tensor_core_schedule": tc_schedule, "cuda_core_tile_columns": simt_tiles or None},
                "e2e": {"value": b.unknowns * world / statistics.median(t_e2e), "unit": UNIT,
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": len(t_e2e),
                        "statistic": "median"},
                "roofline": rooflines[0] if rooflines else None, "rooflines": rooflines, "cpu_baseline": cpu,
                "clocks": clk, "gpu_launches": int(sth.launches), "split_ms_last_step": step_split,
                "host_split_per_step": {"setup_ms": sth.host_setup_ms / a.steps,
                                        "graph_build_ms": sth.graph_build_ms / a.steps,
                                        "cycles_ms": sth.host_cycles_ms / a.steps},
                "variants": variants}
        print(json.dumps(line), flush=True)
    b.close()
    ctx.close()


def run_tbas(a, rank, world, local, dev):
    """The sparse workload: A^(1) = 5-point Laplacian on a 128 x 128 grid, A^(2..8) with 4 random
    entries per row, B dense (s = 32, or --s), solved by TBAS(10) to 1e-10 in FP64.  One step =
    one ts_op_create_csr + ts_tba_solve."""
    import numpy as np
    import torch
    from paper_2405_09233_gb300 import Context, inputs
    cfg = inputs.WORKLOADS["sparse_lap128_s32_p8"]
    s_blk = a.s if a.s is not None else cfg["s"]
    prob = inputs.sparse_problem(grid=cfg["grid"], s=s_blk, p=cfg["p"], seed=rank_seed(rank))
    n, p = prob.n, prob.p
    rowptr, cols, vals, base = [], [], [], 0
    for sl in prob.slices:
        rowptr.append(sl.rowptr.astype(np.int64) + base)
        cols.append(sl.col)
        vals.append(sl.val)
        base += sl.col.size
    rowptr = np.concatenate(rowptr).astype(np.int32)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    ctx = Context(local)
    B_h = torch.from_numpy(inputs.to_device_layout(prob.B)).pin_memory()
    Bd = B_h.to(dev)
    Xs = torch.from_numpy(inputs.to_device_layout(prob.Xstar)).to(dev)
    op0 = ctx.op_create_csr(n, p, rowptr, cols, vals, Bd)
    Cd = ctx.sylv_apply(op0, Xs)
    normC = float(torch.linalg.norm(Cd))
    X = torch.zeros_like(Cd)
    m = 10

    def step(precision=a.precision):
        op = ctx.op_create_csr(n, p, rowptr, cols, vals, Bd)
        X.zero_()
        r = ctx.tba_solve(op, Cd, X, restart=m, tol=1e-10, precision=precision)
        op.close()
        return r

    def certify():
        return float(torch.linalg.norm(Cd - ctx.sylv_apply(op0, X))) / normC

    for _ in range(a.warmup):
        r = step()
        assert r.status == 0, r
    ctx.stats_reset()
    ctx.stats_enable(True)
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.steps):
        r = step()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ctx.stats_enable(False)
    stt = ctx.stats_get()
    ms = max_over_ranks(e0.elapsed_time(e1) / a.steps, dev)
    cert = certify()
    unknowns = n * s_blk * p
    sms = device_sms(dev)
    mhz = clk.get("sm_max_mhz") or peaks()["sm_max_mhz"]
    peak64 = fp64_peak_tflops(sms, mhz)
    probe = measure_fp64_probe(ctx) if rank == 0 else None
    rooflines = []
    if stt.tba_launches:
        blk_ms = stt.tba_ms / stt.tba_launches
        blk_tf = stt.tba_flops / stt.tba_launches / (blk_ms * 1e-3) / 1e12 * 0.75   # 3-multiply form executed
        rooflines.append((stt.tba_ms, {
            "bound": "alu", "achieved": blk_tf, "peak": peak64, "unit": "TFLOP/s", "frac": blk_tf / peak64,
            "traffic": None,
            "kernel": "k_gram / k_rows_mm (TBAS tubal Gram and block update, FP64 complex, n x s blocks)",
            "note": ("FLOPs of the 3-multiply complex form the kernels implement (6 n s^2 per slice product); peak "
                     "derived: 2 DFMA/clk/SM x %d SMs x %.0f MHz. Share of the step: %.3f (timed with events around "
                     "each product)" % (sms, mhz, stt.tba_ms / (ms * a.steps))) + probe_note(probe),
            "peak_probe": probe}))
    if stt.spmm_launches:
        sp_ms = stt.spmm_ms / stt.spmm_launches
        sp_tf = stt.spmm_flops / stt.spmm_launches / (sp_ms * 1e-3) / 1e12
        sp_gbs = stt.spmm_bytes / stt.spmm_launches / (sp_ms * 1e-3) / 1e9
        rooflines.append((stt.spmm_ms, {
            "bound": "alu", "achieved": sp_tf, "peak": peak64, "unit": "TFLOP/s", "frac": sp_tf / peak64,
            "traffic": None,
            "kernel": "k_sylv_rows (complex CSR SpMM over the union pattern, all Fourier slices)",
            "algorithmic_gbs": sp_gbs, "hbm_frac": sp_gbs / peaks()["hbm_gbs"],
            "note": ("FLOPs executed: 8 per stored complex value and block column; peak derived: 2 DFMA/clk/SM x %d "
                     "SMs x %.0f MHz. Algorithmic bytes (values, pattern, V once, W once) / time = %.0f GB/s = %.3f of "
                     "measured HBM. Share of the step: %.3f" % (sms, mhz, sp_gbs, sp_gbs / peaks()["hbm_gbs"],
                                                                stt.spmm_ms / (ms * a.steps))) + probe_note(probe),
            "peak_probe": probe}))
    rooflines.sort(key=lambda t: -t[0])
    rooflines = [r for _, r in rooflines]
    # end to end: B, C and X in host memory (the CSR arrays are host arrays by contract)
    C_h = Cd.cpu().pin_memory()
    X_h = torch.zeros_like(C_h).pin_memory()
    t_e2e = []
    for _ in range(max(a.e2e_steps, 1)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op = ctx.op_create_csr(n, p, rowptr, cols, vals, B_h)
        X_h.zero_()
        r2 = ctx.tba_solve(op, C_h, X_h, restart=m, tol=1e-10, precision=a.precision)
        op.close()
        t_e2e.append(time.perf_counter() - t0)
        assert r2.status == 0, r2
    h2d = 4 * (rowptr.size + cols.size) + 8 * (vals.size + B_h.numel() + 2 * C_h.numel())
    variants = {}
    other = "mixed_fp32" if a.precision == "fp64" else "fp64"
    if a.variants != "":
        try:
            med, msl, rv = timed_median(lambda: step(other), a.reps, 1)
            variants[other] = {"value": unknowns * world / (med / 1e3), "ms_per_step": med, "ms_all": msl,
                               "status": rv.status_name, "cycles": rv.info.cycles, "relres_true": rv.info.relres_true,
                               "relres_fp64_dfma": certify(), "err_vs_xstar": float(torch.max(torch.abs(X - Xs)))}
        except Exception as e:  # report, do not hide
            variants[other] = {"error": str(e)}
    cpu = cpu_baseline_tbas(prob, m) if rank == 0 and world == 1 and not a.no_cpu_baseline else None
    if rank == 0:
        line = {"metric": METRIC, "value": job_throughput(unknowns, world, ms), "unit": UNIT, "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if a.precision == "fp64" else "f32+f64",
                "data": "synthetic",
                "config": {"workload": "sparse_lap128_s32_p8", "n": n, "s": s_blk, "p": p, "restart": m,
                           "precision": a.precision,
                           "tol": 1e-10, "method": "TBAS", "cycles": r.info.cycles, "block_steps": r.info.iters,
                           "relres_true": r.info.relres_true, "relres_fp64_dfma": cert,
                           "err_vs_xstar": float(torch.max(torch.abs(X - Xs))), "sms": sms},
                "e2e": {"value": unknowns * world / statistics.median(t_e2e), "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": 8 * X_h.numel(), "steps": len(t_e2e), "statistic": "median"},
                "roofline": rooflines[0] if rooflines else None, "rooflines": rooflines, "cpu_baseline": cpu,
                "clocks": clk, "gpu_launches": int(stt.launches), "variants": variants}
        print(json.dumps(line), flush=True)
    op0.close()
    ctx.close()


def run_apply_mode(a, ctx, Ad, Bd, Xs, cfg, world, dev):
    """Operator applications only (FP64 ts_sylv_apply, or ts_sylv_apply_lowp): the kernel runs that the
    profiles under profiles/ are taken on.  One step = one application of M."""
    import torch
    n, s, p = cfg["n"], cfg["s"], cfg["p"]
    op = ctx.op_create_dense(Ad, Bd)
    if a.precision == "fp64" and a.engine == "ozaki":
        Xin = Xs
        Y = torch.empty_like(Xs)
        fn = lambda: ctx.sylv_apply_ozaki(op, Xin, Y)  # noqa: E731
    elif a.precision == "fp64":
        Xin = Xs
        Y = torch.empty_like(Xs)
        fn = lambda: ctx.sylv_apply(op, Xin, Y)  # noqa: E731
    else:
        Xin = Xs.float().contiguous()
        Y = torch.empty_like(Xin)
        fn = lambda: ctx.sylv_apply_lowp(op, Xin, a.precision, Y)  # noqa: E731
    for _ in range(a.warmup):
        fn()
    torch.cuda.synchronize()
    ctx.stats_reset()
    ctx.stats_enable(True)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ctx.stats_enable(False)
    st = ctx.stats_get()
    ms = e0.elapsed_time(e1) / a.steps
    sms = device_sms(dev)
    mhz = clk.get("sm_max_mhz") or peaks()["sm_max_mhz"]
    rfs = stats_rooflines(st, n, s, p, ms * a.steps, False, a.precision, sms, mhz, a.workload)
    line = {"mode": "apply", "metric": "operator applications (unknowns/s)", "value": n * s * p / (ms / 1e3),
            "unit": "unknowns/s", "ms_per_step": ms, "steps": a.steps, "warmup": a.warmup,
            "config": {"workload": a.workload, "n": n, "s": s, "p": p, "precision": a.precision,
                       "fp64_engine": a.engine},
            "roofline": rfs[0] if rfs else None, "rooflines": rfs,
            "fft_gbs": st.fft_bytes / max(st.fft_ms, 1e-9) / 1e6,
            "fft_ms_per_step": st.fft_ms / a.steps, "clocks": clk, "gpu_launches": int(st.launches)}
    print(json.dumps(line), flush=True)
    op.close()
    ctx.close()


if __name__ == "__main__":
    main()
