#!/usr/bin/env python3
"""Benchmark: Sylvester-tensor-equation unknowns solved per second, to a true relative residual
of 1e-10, on GB300.

One step = one complete solve of A*X - X*B = C from X0 = 0 through the C ABI (operator setup
ts_op_create_dense included), with the inputs resident in HBM.  The default workload is the
dense 1024 x 1024 x 16 family (A^(1) = tridiag(-1,4,-1) + 0.1 G/sqrt(n), ...; X* ~ U(-1,1),
C = M(X*)) solved by FP64 tGMRES(30).  Every rank solves its own instance (weak scaling, no
collective on the data path).

The JSON line also carries: `e2e` (the same metric with host buffers, copies inside the timed
region), `roofline` for the dominant kernel (the per-slice GEMM, timed by CUDA events inside
the library over the timed region), `cpu_baseline` (the CPU oracle on this host's cores, on a
bounded sample), `clocks` sampled during the timed region, `gpu_launches`, and `variants`
(mixed precision on the same workload).
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
FP64_NOMINAL_TFLOPS = 4 * 152 * 2.070e9 / 1e12   # 4 FP64 FLOP/clk/SM x 152 SMs x 2070 MHz


def args_parse():
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
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", choices=["solve", "apply"], default="solve",
                    help="solve: full solves (the benchmark); apply: operator applications only (kernel runs)")
    ap.add_argument("--count", type=int, default=None, help="instances of the batched workload (default 256)")
    ap.add_argument("--n", type=int)
    ap.add_argument("--s", type=int)
    ap.add_argument("--p", type=int)
    return ap.parse_args()


DENSE_VARIANTS = "tfom,mixed_fp32,mixed_tf32x3,mixed_tf32,mixed_bf16,fp64@ozaki,tfom@ozaki,mixed_tf32x3@ozaki,mixed_bf16@ozaki"
BATCHED_VARIANTS_DEFAULT_MARK = "<batched-default>"


def workload_cfg(a):
    from paper_2405_09233_gb300 import inputs
    cfg = dict(inputs.WORKLOADS[a.workload])
    for key in ("n", "s", "p"):
        if getattr(a, key) is not None:
            cfg[key] = getattr(a, key)
    return cfg


def peaks():
    """Roofline denominators: MEASURED_PEAKS.json when present, else the recipe's fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_burst": d["bf16_tflops"], "bf16_sustained": d["bf16_tflops_sustained"],
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_burst": 1900.0, "bf16_sustained": 1700.0, "source": "fallback"}


TF32_OVER_BF16 = 1.1 / 2.25       # nominal dense tensor rates (PFLOP/s per GPU)
FFMA_NOMINAL_TFLOPS = 2 * 128 * 152 * 2.070e9 / 1e12   # 128 FP32 lanes/SM x 2 FLOP x 152 SMs x 2070 MHz


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the dominant kernels at the
# n = s = 1024, p = 16 workload, from one ncu capture each (profiles/traffic_dense_n1024_s1024_p16.md);
# a roofline object carries them only for that workload and, for the emulated product, only when every
# launch used 6 digits.
TRAFFIC_N1024 = {"k_gemm_slices<double>": 497799168 + 137544960, "k_oz_sylv/6": 1779147520 + 149931264}


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
            "note": "peak: %s BF16 %s; FP64-equivalent rate %.2f TFLOP/s. Kernel share of the step: %.3f"
                    % (pk["source"], "sustained" if sustained else "burst",
                       flops_per_launch / (avg_ms * 1e-3) / 1e12, share)}


def gemm_roofline(kind, precision, flops_per_launch, avg_ms, sustained, share):
    """Roofline object for the dominant slice-GEMM kernel."""
    achieved = flops_per_launch / (avg_ms / 1e3) / 1e12
    pk = peaks()
    if kind == "fp64":
        return {"bound": "alu", "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_NOMINAL_TFLOPS, "traffic": None,
                "kernel": "k_gemm_slices<double> (FP64 DFMA, 3-multiply complex)",
                "note": ("peak derived: 4 FP64 FLOP/clk/SM x 152 SMs x 2070 MHz (nominal). Algorithmic FLOPs count 8 "
                         "per complex multiply-add; the kernel executes 6 (Gauss), so frac can reach 1.33. "
                         f"Kernel share of the step: {share:.3f}")}
    if precision == "mixed_fp32":
        return {"bound": "alu", "achieved": achieved, "peak": FFMA_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FFMA_NOMINAL_TFLOPS, "traffic": None,
                "kernel": "k_gemm_slices<float> (FP32 FFMA, 3-multiply complex)",
                "note": f"peak derived: 2 FLOP x 128 lanes/SM x 152 SMs x 2070 MHz. Kernel share: {share:.3f}"}
    bf = pk["bf16_sustained"] if sustained else pk["bf16_burst"]
    tf32 = precision in ("mixed_tf32", "mixed_tf32x3")
    parts = 3 if precision == "mixed_tf32x3" else 1
    peak = bf * (TF32_OVER_BF16 if tf32 else 1.0) / parts
    name = {"mixed_tf32": "TF32", "mixed_bf16": "BF16", "mixed_tf32x3": "split TF32 x3"}[precision]
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": f"k_tc_sylv ({name} tcgen05)",
            "note": (f"peak: {pk['source']} BF16 {'sustained' if sustained else 'burst'}"
                     + (" x nominal TF32/BF16 ratio 0.489" if tf32 else "")
                     + (" / 3 products (split TF32)" if parts == 3 else "")
                     + f". Kernel share of the step: {share:.3f}")}


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


# ------------------------------------------------------------------------------------------------
# the CPU oracle on a bounded sample (rank 0, N = 1)
# ------------------------------------------------------------------------------------------------
def oracle_apply_sample(wl_cfg, seed, n_applies=2):
    """Time n_applies oracle applications of M (Definition 2.1 route) at the full workload size."""
    import numpy as np
    from paper_2405_09233_gb300 import inputs
    from oracle import krylov
    pr = inputs.dense_problem(wl_cfg["n"], wl_cfg["s"], wl_cfg["p"], seed=seed, scale=wl_cfg["scale"])
    X = pr.Xstar
    times = []
    for _ in range(n_applies):
        t0 = time.perf_counter()
        Y = krylov.sylv_apply(pr.A, pr.B, X)
        times.append(time.perf_counter() - t0)
        X = Y / np.linalg.norm(Y)
    return min(times)


def oracle_applies_needed(wl_cfg, seed):
    """Operator applications the oracle's own tGMRES needs on the same family at n = s = 128
    (the spectrum of this family, hence the iteration count, does not depend on n)."""
    from paper_2405_09233_gb300 import inputs
    from oracle import krylov
    pr = inputs.dense_problem(128, 128, wl_cfg["p"], seed=seed, scale=wl_cfg["scale"])
    C = krylov.sylv_apply(pr.A, pr.B, pr.Xstar)
    r = krylov.tgmres(pr.A, pr.B, C, m=wl_cfg["restart"], tol=1e-10)
    return r.iters + r.cycles + 1, r


def cpu_baseline(wl_cfg, seed):
    import numpy as np
    n, s, p = wl_cfg["n"], wl_cfg["s"], wl_cfg["p"]
    t_apply = oracle_apply_sample(wl_cfg, seed)
    applies, r = oracle_applies_needed(wl_cfg, seed)
    t_solve = t_apply * applies
    cores = os.cpu_count()
    return {"value": n * s * p / t_solve, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"oracle M(X) (bcirc block-row definition, numpy FP64, {cores} host threads) timed at "
                       f"n={n}, s={s}, p={p}: {t_apply:.2f} s/apply; x {applies} applies (the oracle tGMRES("
                       f"{wl_cfg['restart']}) iteration count + residuals at n=s=128, same family); "
                       f"MGS cost (<1%) not included")}


# ------------------------------------------------------------------------------------------------
def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2405_09233_gb300 import inputs
    cfg = inputs.WORKLOADS[a.workload]
    n, s, p = cfg["n"], cfg["s"], cfg["p"]
    applies, _ = oracle_applies_needed(cfg, 1)
    for _ in range(a.warmup):
        oracle_apply_sample(cfg, 1, n_applies=1)
    ts = []
    for _ in range(a.steps):
        ts.append(oracle_apply_sample(cfg, 1, n_applies=1))
    t_step = statistics.mean(ts)
    value = n * s * p / (t_step * applies)
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_step * applies * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": a.workload, "n": n, "s": s, "p": p,
                                            "restart": cfg["restart"], "tol": 1e-10},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step = one oracle M(X) at full size ({t_step:.2f} s); "
                                       f"solve time = step x {applies} applies (oracle tGMRES count at n=s=128)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = args_parse()
    if a.variants is None:
        a.variants = BATCHED_VARIANTS_DEFAULT_MARK if a.workload == "batched_256" else DENSE_VARIANTS
    if a.precision is None:
        a.precision = ("fp64" if a.workload in ("dense_n24_s24_p4", "dense_n1024_s1024_p16", "sparse_lap128_s32_p8")
                       else "mixed_fp32")
    if a.impl == "reference":
        run_reference(a)
        return
    import numpy as np
    import torch
    from paper_2405_09233_gb300 import Context, inputs

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
    cfg = workload_cfg(a)
    n, s, p, m = cfg["n"], cfg["s"], cfg["p"], cfg["restart"]
    seed = rank_seed(rank)
    pr = inputs.dense_problem(n, s, p, seed=seed, scale=cfg["scale"])
    A_h = torch.from_numpy(inputs.to_device_layout(pr.A)).pin_memory()
    B_h = torch.from_numpy(inputs.to_device_layout(pr.B)).pin_memory()
    Xs_h = torch.from_numpy(inputs.to_device_layout(pr.Xstar)).pin_memory()
    Ad, Bd, Xs = A_h.to(dev), B_h.to(dev), Xs_h.to(dev)
    ctx = Context(local)
    op0 = ctx.op_create_dense(Ad, Bd)
    Cd = ctx.sylv_apply(op0, Xs)              # manufactured right-hand side C = M(X*)
    op0.close()
    X = torch.zeros_like(Cd)
    torch.cuda.synchronize()
    if a.mode == "apply":
        return run_apply_mode(a, ctx, Ad, Bd, Xs, cfg, world, dev)

    def step(precision, engine=a.engine):
        op = ctx.op_create_dense(Ad, Bd)
        X.zero_()
        if precision == "tfom":   # restarted tFOM(m), FP64 (variant)
            r = ctx.tfom_solve(op, Cd, X, restart=m, tol=1e-10, engine=engine)
        else:
            r = ctx.tgmres_solve(op, Cd, X, restart=m, tol=1e-10, precision=precision, engine=engine)
        op.close()
        return r

    for _ in range(a.warmup):
        r = step(a.precision)
    assert r.status == 0, r

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    ctx.stats_reset()
    ctx.stats_enable(True)
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    ev0.record()
    results = [step(a.precision) for _ in range(a.steps)]
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ctx.stats_enable(False)
    st = ctx.stats_get()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / a.steps, dev)
    last = results[-1]
    assert all(r.status == 0 for r in results), results
    relres = last.info.relres_true
    err_xstar = float(torch.max(torch.abs(X - Xs)) / torch.max(torch.abs(Xs)))
    unknowns = n * s * p
    value = job_throughput(unknowns, world, ms)

    # dominant kernel: whichever slice-GEMM class (FP64 DFMA, emulated FP64, low precision) took most time
    step_ms_total = ms * a.steps
    top = max(("fp64", st.gemm_ms), ("oz", st.oz_ms), ("lowp", st.lowp_ms), key=lambda t: t[1])[0]
    if top == "fp64":
        roofline = gemm_roofline("fp64", "fp64", st.gemm_flops / max(st.gemm_launches, 1),
                                 st.gemm_ms / max(st.gemm_launches, 1), True, st.gemm_ms / step_ms_total)
        roofline["traffic"] = traffic_for("k_gemm_slices<double>", a.workload)
    elif top == "oz":
        roofline = ozaki_roofline(st.oz_flops / max(st.oz_launches, 1), st.oz_pair_flops / max(st.oz_launches, 1),
                                  st.oz_ms / max(st.oz_launches, 1),
                                  True, st.oz_ms / step_ms_total)
        if abs(st.oz_pair_flops - 21 * st.oz_flops) <= 1e-9 * st.oz_pair_flops:   # 6 digits in every launch
            roofline["traffic"] = traffic_for("k_oz_sylv/6", a.workload)
    else:
        roofline = gemm_roofline("lowp", a.precision, st.lowp_flops / max(st.lowp_launches, 1),
                                 st.lowp_ms / max(st.lowp_launches, 1), True, st.lowp_ms / step_ms_total)
    kernel_times = {"fp64_gemm_ms": st.gemm_ms / a.steps, "ozaki_gemm_ms": st.oz_ms / a.steps,
                    "lowp_gemm_ms": st.lowp_ms / a.steps,
                    "fft_ms": st.fft_ms / a.steps, "fp64_gemm_launches": st.gemm_launches // a.steps,
                    "ozaki_gemm_launches": st.oz_launches // a.steps,
                    "lowp_gemm_launches": st.lowp_launches // a.steps,
                    "fft_gbs": st.fft_bytes / max(st.fft_ms, 1e-9) / 1e6}

    # end to end through the C ABI with host buffers (copies inside the timed region)
    C_h = Cd.cpu().pin_memory()
    X_h = torch.zeros_like(C_h).pin_memory()
    e2e_times, e2e_parts = [], []
    for _ in range(max(a.e2e_steps, 0)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op = ctx.op_create_dense(A_h, B_h)
        t1 = time.perf_counter()
        X_h.zero_()
        r = ctx.tgmres_solve(op, C_h, X_h, restart=m, tol=1e-10, precision=a.precision, engine=a.engine)
        t2 = time.perf_counter()
        op.close()
        t3 = time.perf_counter()
        e2e_times.append(t3 - t0)
        e2e_parts.append((t1 - t0, t2 - t1, t3 - t2))
        assert r.status == 0, r
    e2e = {"value": unknowns * world / statistics.median(e2e_times) if e2e_times else None, "unit": UNIT,
           "h2d_bytes_per_step": 8 * (n * n * p + s * s * p + 2 * n * s * p),
           "d2h_bytes_per_step": 8 * n * s * p}
    if e2e_parts:   # host-clock split of the last end-to-end step: operator setup, solve, release
        e2e["split_ms"] = dict(zip(("op_create", "solve", "op_destroy"), (round(x * 1e3, 3) for x in e2e_parts[-1])))

    variants = {}
    primary = a.precision + ("" if a.engine == "dfma" else "@" + a.engine)
    for name in [v for v in a.variants.split(",") if v and v != primary]:
        prec, _, eng = name.partition("@")
        eng = eng or "dfma"
        try:
            step(prec, eng)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            rv = step(prec, eng)
            e1.record()
            torch.cuda.synchronize()
            tv = e0.elapsed_time(e1)
            variants[name] = {"value": unknowns * world / (tv / 1e3), "ms_per_step": tv,
                              "status": rv.status_name, "relres_true": rv.info.relres_true,
                              "outer": rv.info.outer, "inner_iters": rv.info.iters,
                              "applies_fp64": rv.info.applies_fp64, "applies_low": rv.info.applies_low,
                              "err_vs_xstar": float(torch.max(torch.abs(X - Xs)) / torch.max(torch.abs(Xs)))}
        except Exception as e:  # report, do not hide
            variants[name] = {"error": str(e)}

    if n * s * p <= 1 << 16:
        # small problems are launch-latency bound: also time the graph-replayed form (the batched
        # solver on this single instance: one CUDA graph per restart cycle, no per-step host sync)
        try:
            ops1 = [ctx.op_create_dense(Ad, Bd)]
            for _ in range(3):
                X.zero_()
                ctx.batched_solve(ops1, [Cd], [X], restart=m, tol=1e-10, precision=a.precision)
            torch.cuda.synchronize()
            reps = 20
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                X.zero_()
                stb, infb, _ = ctx.batched_solve(ops1, [Cd], [X], restart=m, tol=1e-10, precision=a.precision)
            e1.record()
            torch.cuda.synchronize()
            tb = e0.elapsed_time(e1) / reps
            variants["graph_replay"] = {"value": unknowns * world / (tb / 1e3), "ms_per_step": tb, "status": stb,
                                        "inner_iters": infb[0].iters, "relres_true": infb[0].relres_true,
                                        "us_per_inner_step": 1e3 * tb / max(infb[0].iters, 1)}
            ops1[0].close()
        except Exception as e:  # report, do not hide
            variants["graph_replay"] = {"error": str(e)}
        variants["us_per_inner_step"] = 1e3 * ms / max(last.info.iters, 1)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline and a.workload == "dense_n1024_s1024_p16":
        cpu = cpu_baseline(cfg, seed)

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
                           "applies_fp64": last.info.applies_fp64, "relres_true": relres,
                           "err_vs_xstar": err_xstar},
                "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu, "clocks": clk,
                "gpu_launches": int(st.launches), "kernels_per_step": kernel_times, "variants": variants}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batched(a, rank, world, local, dev):
    """The batched workload: 256 instances (n log-uniform in [64, 1024], s uniform in [16, 128],
    p in {4, 8, 16}), one step = one ts_batched_solve of all of them (operator setup included)."""
    import torch
    from paper_2405_09233_gb300 import Context, inputs
    count = a.count if a.count else inputs.WORKLOADS["batched_256"]["count"]
    specs = inputs.batched_specs(count, seed=4 + rank)
    ctx = Context(local)
    host = []
    for sp in specs:
        pr = inputs.dense_problem(sp.n, sp.s, sp.p, seed=sp.seed)
        host.append((torch.from_numpy(inputs.to_device_layout(pr.A)).pin_memory(),
                     torch.from_numpy(inputs.to_device_layout(pr.B)).pin_memory(),
                     torch.from_numpy(inputs.to_device_layout(pr.Xstar)).pin_memory()))
    dev_in = [(A.to(dev), B.to(dev), X.to(dev)) for A, B, X in host]
    Cs = []
    for A, B, Xst in dev_in:
        op = ctx.op_create_dense(A, B)
        Cs.append(ctx.sylv_apply(op, Xst))
        op.close()
    Xs = [torch.zeros_like(C) for C in Cs]
    unknowns = sum(sp.n * sp.s * sp.p for sp in specs)
    prec = a.precision

    def step(precision, engine=a.engine):
        ops = [ctx.op_create_dense(A, B) for A, B, _ in dev_in]
        for X in Xs:
            X.zero_()
        st, infos, sts = ctx.batched_solve(ops, Cs, Xs, restart=20, tol=1e-10, precision=precision, engine=engine)
        for op in ops:
            op.close()
        return st, infos

    for _ in range(a.warmup):
        st, infos = step(prec)
    assert st == 0
    ctx.stats_reset()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.steps):
        st, infos = step(prec)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    stt = ctx.stats_get()
    ms = max_over_ranks(e0.elapsed_time(e1) / a.steps, dev)
    relres = max(i.relres_true for i in infos)
    err = max(float(torch.max(torch.abs(X - Xst))) for X, (_, _, Xst) in zip(Xs, dev_in))
    # end to end: operators and right-hand sides from pinned host memory, solutions back to host
    C_h = [C.cpu().pin_memory() for C in Cs]
    X_h = [torch.zeros_like(C) for C in C_h]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ops = [ctx.op_create_dense(A, B) for A, B, _ in host]
    Cd = [C.to(dev, non_blocking=True) for C in C_h]
    Xd = [torch.zeros_like(C) for C in Cd]
    st2, _, _ = ctx.batched_solve(ops, Cd, Xd, restart=20, tol=1e-10, precision=prec, engine=a.engine)
    for Xh_, Xd_ in zip(X_h, Xd):
        Xh_.copy_(Xd_)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    for op in ops:
        op.close()
    h2d = sum(8 * (A.numel() + B.numel() + C.numel()) for (A, B, _), C in zip(host, C_h))
    d2h = sum(8 * X.numel() for X in X_h)
    variants = {}
    primary = prec + ("" if a.engine == "dfma" else "@" + a.engine)
    names = a.variants.split(",") if a.variants else []
    if a.variants == BATCHED_VARIANTS_DEFAULT_MARK:
        names = ["fp64", "mixed_fp32", "fp64@ozaki", "mixed_fp32@ozaki", "mixed_tf32x3@ozaki", "mixed_bf16@ozaki"]
    for name in [v for v in names if v and v != primary]:
        vp, _, ve = name.partition("@")
        try:
            torch.cuda.synchronize()
            f0 = time.perf_counter()
            stf, infof = step(vp, ve or "dfma")
            torch.cuda.synchronize()
            variants[name] = {"value": unknowns * world / (time.perf_counter() - f0), "status": stf,
                              "max_relres_true": max(i.relres_true for i in infof),
                              "max_err_vs_xstar": max(float(torch.max(torch.abs(X - Xst)))
                                                      for X, (_, _, Xst) in zip(Xs, dev_in))}
        except Exception as e:  # report, do not hide
            variants[name] = {"error": str(e)}
    if rank == 0:
        line = {"metric": METRIC, "value": unknowns * world / (ms / 1e3), "unit": UNIT, "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64" if prec != "fp64" else "f64", "data": "synthetic",
                "config": {"workload": "batched_256" if count == 256 else "batched_%d" % count, "instances": count,
                           "unknowns": unknowns, "restart": 20,
                           "tol": 1e-10, "precision": prec, "fp64_engine": a.engine, "method": "batched tGMRES",
                           "max_relres_true": relres, "max_err_vs_xstar": err,
                           "l2": "inputs larger than L2 (5 GB basis)"},
                "e2e": {"value": unknowns * world / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "clocks": clk, "gpu_launches": int(stt.launches), "variants": variants}
        print(json.dumps(line), flush=True)
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
    Bd = torch.from_numpy(inputs.to_device_layout(prob.B)).to(dev)
    Xs = torch.from_numpy(inputs.to_device_layout(prob.Xstar)).to(dev)
    op0 = ctx.op_create_csr(n, p, rowptr, cols, vals, Bd)
    Cd = ctx.sylv_apply(op0, Xs)
    op0.close()
    X = torch.zeros_like(Cd)
    m = 10

    def step(precision=a.precision):
        op = ctx.op_create_csr(n, p, rowptr, cols, vals, Bd)
        X.zero_()
        r = ctx.tba_solve(op, Cd, X, restart=m, tol=1e-10, precision=precision)
        op.close()
        return r

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
    unknowns = n * s_blk * p
    blk_ms = stt.tba_ms / max(stt.tba_launches, 1)
    blk_tf = stt.tba_flops / max(stt.tba_launches, 1) / (blk_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": blk_tf, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "frac": blk_tf / FP64_NOMINAL_TFLOPS, "traffic": None,
                "kernel": "k_gram / k_rows_mm (TBAS tubal Gram and block update, FP64 complex, n x s blocks)",
                "note": ("peak derived: 4 FP64 FLOP/clk/SM x 152 SMs x 2070 MHz (nominal); 8 n s^2 FLOP per slice "
                         "product. Share of the step: %.3f (timed with events around each product, which adds "
                         "event overhead)" % (stt.tba_ms / (ms * a.steps)))}
    variants = {}
    other = "mixed_fp32" if a.precision == "fp64" else "fp64"
    if a.variants != "":
        try:
            step(other)
            torch.cuda.synchronize()
            v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            v0.record()
            rv = step(other)
            v1.record()
            torch.cuda.synchronize()
            tv = v0.elapsed_time(v1)
            variants[other] = {"value": unknowns * world / (tv / 1e3), "ms_per_step": tv, "status": rv.status_name,
                               "cycles": rv.info.cycles, "relres_true": rv.info.relres_true,
                               "err_vs_xstar": float(torch.max(torch.abs(X - Xs)))}
        except Exception as e:  # report, do not hide
            variants[other] = {"error": str(e)}
    if rank == 0:
        line = {"metric": METRIC, "value": job_throughput(unknowns, world, ms), "unit": UNIT, "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if a.precision == "fp64" else "f32+f64",
                "data": "synthetic",
                "config": {"workload": "sparse_lap128_s32_p8", "n": n, "s": s_blk, "p": p, "restart": m,
                           "precision": a.precision,
                           "tol": 1e-10, "method": "TBAS", "cycles": r.info.cycles, "block_steps": r.info.iters,
                           "relres_true": r.info.relres_true,
                           "err_vs_xstar": float(torch.max(torch.abs(X - Xs)))},
                "roofline": roofline, "clocks": clk, "gpu_launches": int(stt.launches), "variants": variants}
        print(json.dumps(line), flush=True)
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
    if a.precision == "fp64" and a.engine == "ozaki":
        rf = ozaki_roofline(st.oz_flops / max(st.oz_launches, 1), st.oz_pair_flops / max(st.oz_launches, 1),
                                  st.oz_ms / max(st.oz_launches, 1), False,
                            st.oz_ms / (ms * a.steps))
    elif a.precision == "fp64":
        rf = gemm_roofline("fp64", "fp64", st.gemm_flops / max(st.gemm_launches, 1),
                           st.gemm_ms / max(st.gemm_launches, 1), False, st.gemm_ms / (ms * a.steps))
    else:
        rf = gemm_roofline("lowp", a.precision, st.lowp_flops / max(st.lowp_launches, 1),
                           st.lowp_ms / max(st.lowp_launches, 1), False, st.lowp_ms / (ms * a.steps))
    line = {"mode": "apply", "metric": "operator applications (unknowns/s)", "value": n * s * p / (ms / 1e3),
            "unit": "unknowns/s", "ms_per_step": ms, "steps": a.steps, "warmup": a.warmup,
            "config": {"workload": a.workload, "n": n, "s": s, "p": p, "precision": a.precision,
                       "fp64_engine": a.engine},
            "roofline": rf, "fft_gbs": st.fft_bytes / max(st.fft_ms, 1e-9) / 1e6,
            "fft_ms_per_step": st.fft_ms / a.steps, "clocks": clk, "gpu_launches": int(st.launches)}
    print(json.dumps(line), flush=True)
    op.close()
    ctx.close()


if __name__ == "__main__":
    main()
