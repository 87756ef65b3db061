#!/usr/bin/env python
"""Benchmark of the GB300 Jacobi solver on the single large dense system.

Workload: n = 16384, one right-hand side, strictly diagonally dominant A (off-diagonals uniform [-1, 1),
a_ii = 1.05 * sum_{j != i} |a_ij| * (random sign), so ||T||_inf = 1/1.05), planted X* uniform [-1, 1),
B = A X*, X0 = 0, target ||B - A X||_inf / ||B||_inf <= 1e-10.  Inputs are synthetic and seeded
(``synth``), resident in HBM before the timed region; A (2.15 GB) is far larger than the 129 MB L2, so
no flush is needed between steps.

One step = one complete solve through the C ABI: ``jacobi_setup_ex`` (diagonal check, 1/a_ii, the narrow
copy of A for the mixed paths) + ``jacobi_solve_async`` (one persistent kernel).  The headline path is
BF16 inner sweeps with FP64 iterative refinement; the plain FP64 Jacobi path and the E4M3 path are timed
the same way beside it.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle instead (the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s at ||AX-B||/||B||<=1e-10 (BF16 inner sweeps + FP64 refinement), n=16384"
TARGET = 1e-10
ESIZE = {"fp64": 8, "fp32_ir": 4, "bf16_ir": 2, "fp8_ir": 1}
PATH_LABEL = {"bf16_ir": "BF16 inner sweeps + FP64 refinement to rel. residual 1e-10",
              "fp8_ir": "FP8 (E4M3) inner sweeps + FP64 refinement to rel. residual 1e-10",
              "fp32_ir": "FP32 inner sweeps + FP64 refinement to rel. residual 1e-10",
              "fp64": "FP64 Jacobi sweeps to max|dx| < 1e-12",
              "fp64+gs": "FP64 chained Gauss-Seidel sweeps to max|dx| < 1e-12"}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
# each timed kernel's translation unit and every header it includes (the solve kernels share one)
SOLVE_SRC = [os.path.join(ROOT, "paper_1403_5805_gb300", "csrc", f)
             for f in ("solve.cu", "solver.cuh", "dot.cuh", "device_util.cuh", "splitfloat.cuh")]
KERNEL_SRC = {"gs_solve_kernel": [os.path.join(ROOT, "paper_1403_5805_gb300", "csrc", f)
                                  for f in ("gs.cu", "gs.cuh", "solver.cuh", "device_util.cuh")]}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def src_hash(kernel: str = ""):
    h = hashlib.sha256()
    for path in KERNEL_SRC.get(kernel, SOLVE_SRC):
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str, n: int):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current kernel source and
    the same system size."""
    try:
        with open(TRAFFIC_FILE) as fh:
            t = json.load(fh)
    except OSError:
        return None
    e = t.get(kernel)
    if not e or e.get("source_sha256_16") != src_hash(kernel) or e.get("n") != n:
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during a timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.rows = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "20",
                 "-i", str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.proc.stdout.readline()  # wait until sampling runs
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------------------------- our arm

def run_ours(args, world, rank, local):
    import torch

    import synth
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    import paper_1403_5805_gb300 as jac

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if args.only == "mrhs":
        return {"section": "many_rhs", **run_many_rhs(args, jac, torch, dev)}
    if args.only == "batch":
        return {"section": "batched", **run_batch(args, jac, torch, dev)}
    if args.only == "sparse":
        return {"section": "sparse", **run_sparse(args, jac, torch, dev)}
    if args.only == "serve":
        return {"section": "serving", **run_serve(args, jac, torch, dev, args.serve_seconds)}
    if args.only == "small":
        return {"section": "small_system", **run_small(args, jac, torch, dev)}
    if args.only == "sym":
        return {"section": "symmetric", **run_symmetric(args, jac, torch, dev)}
    n, f = args.n, args.f
    A, B, Xs = synth.dominant_system(n, f, seed=synth.BASE_SEED + 1)
    At = torch.from_numpy(A).to(dev)
    Bt = torch.from_numpy(B[:, 0].copy()).to(dev)
    stream = torch.cuda.current_stream(dev)
    ws = torch.empty(0, dtype=torch.uint8, device=dev)
    out = torch.empty(n, dtype=torch.float64, device=dev)
    Xs_t = torch.from_numpy(Xs[:, 0].copy()).to(dev)

    def one_step(prec, ev=None):
        nonlocal ws
        split = prec.endswith("+split") or (args.split_residual and not prec.startswith("fp64"))
        method = "sor" if prec.endswith("+gs") else "jacobi"
        s = jac.DeviceSolver(At, Bt, precision=prec.replace("+split", "").replace("+gs", ""),
                             workspace=ws if ws.numel() else None, inner_rtol=args.inner_rtol,
                             max_inner=args.max_inner, split_residual=split, method=method)
        ws = s.workspace
        if ev is not None:
            ev[0].record(stream)
        s.solve_async(None, args.max_iter, TARGET if not prec.startswith("fp64") else args.fp64_tol, out)
        if ev is not None:
            ev[1].record(stream)
        return s

    xs_host = {}

    def timed(prec, steps, warmup, sample_clocks=False):
        for _ in range(warmup):
            s = one_step(prec)
        torch.cuda.synchronize(dev)
        launch_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                     for _ in range(steps)]
        sampler = ClockSampler(local) if sample_clocks else None
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(steps):
            s = one_step(prec, launch_ev[k])
        t1.record(stream)
        torch.cuda.synchronize(dev)
        clocks = sampler.stop() if sampler else None
        ms = t0.elapsed_time(t1)
        kernel_ms = sum(a.elapsed_time(b) for a, b in launch_ev) / steps
        st = s.last_stats()
        rel = s.residual(out)
        err = float((out - Xs_t).abs().max().item())
        xs_host[prec] = out.cpu().numpy().copy()  # for the error against the oracle's solution
        return {"ms_total": ms, "kernel_ms": kernel_ms, "stats": st.as_dict(), "rel_residual_check": rel,
                "err_vs_xstar": err, "clocks": clocks, "phases": phase_bandwidth(s.trace(), n, prec)}

    main = timed(args.precision, args.steps, args.warmup, sample_clocks=True)
    ms_step = main["ms_total"] / args.steps
    ms_max, value = job_rate(ms_step, world, dev)

    # algorithmic bytes of the dominant kernel (the persistent solve kernel) per launch
    st = main["stats"]
    es = ESIZE[args.precision.replace("+gs", "")]
    outer_with_matrix = max(st["outer_steps"] - 1, 0)  # X0 = 0: the first residual needs no matrix pass
    bytes_launch = outer_with_matrix * 8.0 * n * n + st["sweeps"] * es * float(n) * n
    fused = "narrow_inner" in main["phases"]  # that sweep also reads FP64 A (and writes the narrow copy)
    if fused:
        bytes_launch += 8.0 * n * n
    peaks, peak_kind = measured_peaks()
    achieved = bytes_launch / (main["kernel_ms"] * 1e-3) / 1e9
    kname = {"bf16_ir": "ir_solve_kernel<__nv_bfloat16>", "fp8_ir": "ir_solve_kernel<__nv_fp8_e4m3>",
             "fp32_ir": "ir_solve_kernel<float>", "fp64": "fp64_solve_kernel",
             "fp64+gs": "gs_solve_kernel"}[args.precision]
    traffic = committed_traffic(kname, n)
    roofline = {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                "algorithmic_bytes_per_launch": bytes_launch, "kernel_ms": round(main["kernel_ms"], 4),
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback"}

    fma = fma_peaks(jac, torch, dev)
    composite = composite_roofline(main, n, args.precision, peaks, dev, torch, fma)
    paths = {args.precision: summarize(main, args.steps, n, args.precision)}
    if not args.quick:
        for prec in [p for p in ("fp64", "fp64+gs", "fp8_ir", "fp32_ir", "bf16_ir+split", "fp32_ir+split")
                     if p != args.precision]:
            paths[prec] = summarize(timed(prec, args.steps, args.warmup), args.steps, n, prec)
    fp64_ratio = None
    if "fp64" in paths:
        fp64_ratio = round(paths[args.precision]["solves_per_s"] / paths["fp64"]["solves_per_s"], 3)

    e2e = None if args.no_e2e else run_e2e(args, jac, torch, dev, A, B, ws)
    cpu, x_oracle = (cpu_baseline(A, B, n) if (rank == 0 and world == 1 and not args.no_cpu_baseline)
                     else (None, None))
    err_vs_oracle = None
    if x_oracle is not None:
        # every path's X against the oracle's FP64 Jacobi solution of the same system (relative max-norm)
        scale = float(np.max(np.abs(x_oracle)))
        for prec, x in xs_host.items():
            if prec in paths:
                paths[prec]["err_vs_oracle"] = float(np.max(np.abs(x - x_oracle)) / scale)
        err_vs_oracle = paths[args.precision].get("err_vs_oracle")
    hard = None if (args.quick or args.no_hard) else run_hard(args, jac, torch, dev, ws)
    small = None if (args.quick or args.no_small) else run_small(args, jac, torch, dev)
    batched = None if (args.quick or args.no_batch) else run_batch(args, jac, torch, dev)
    del At, Bt, A, B  # free the single-system inputs before the large many-right-hand-side workload
    many_rhs = None if (args.quick or args.no_mrhs) else run_many_rhs(args, jac, torch, dev)
    sparse = None if (args.quick or args.no_sparse) else run_sparse(args, jac, torch, dev)
    serving = None if (args.quick or args.no_serve) else run_serve(args, jac, torch, dev, args.serve_seconds,
                                                                      args.serve_window)
    result = {
        "metric": METRIC if (args.precision == "bf16_ir" and n == 16384)
        else f"solves/s ({PATH_LABEL[args.precision]}), n={n}",
        "value": round(value, 3), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"bf16_ir": "bf16", "fp64+gs": "fp64"}.get(args.precision, args.precision),
        "data": "synthetic (seeded Philox4x32-10), resident in HBM",
        "config": {"workload": f"single dense system n={n}, f={f}, 1 RHS, {PATH_LABEL[args.precision]}; "
                               f"one step = setup + solve",
                   "n": n, "dominance": f, "nrhs": 1, "precision": args.precision, "global_batch": world,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": f"inputs ({8 * n * n / 1e9:.2f} GB A) larger than the 129 MB L2; no flush"
                         if 8 * n * n > 129e6 else "A fits in the 129 MB L2 (small case; not the bench workload)"},
        # per step: diagonal check, right-hand side, (narrow copy,) solve; BF16 / FP32 inner sweeps write
        # their narrow copy inside the solve kernel
        "gpu_launches": (3 if args.precision.startswith("fp64") or fused else 4) * args.steps,
        "clocks": main["clocks"], "roofline": roofline, "roofline_composite": composite, "fma_peaks": fma,
        "paths": paths,
        "err_vs_oracle": err_vs_oracle,
        "mixed_vs_fp64_solves_ratio": fp64_ratio, "e2e": e2e, "batched": batched, "many_rhs": many_rhs,
        "sparse": sparse,
        "serving": serving, "hard_generator": hard, "small_system": small,
    }
    if cpu is not None:
        result["cpu_baseline"] = cpu
    return result


def job_rate(ms_step, world, device):
    """Replicas: every rank solves its own system per step, so the job's step time is the slowest rank's
    (a MAX all-reduce over the process group) and the job's rate is world / that time.  Returns
    (ms per step, solves per second)."""
    ms_max = ms_step
    if world > 1:
        import torch
        t = torch.tensor([ms_step], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_max = float(t.item())
    return ms_max, world / (ms_max * 1e-3)


def fma_peaks(jac, torch, dev):
    """FP64 and FP32 FMA rates of this GPU's CUDA cores, measured here (jacobi_measure_fma_rates), beside
    the rate derived from the unit count (2 FP64 FMA per clock per SM at the maximum SM clock)."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    f64, f32 = jac.measure_fma_rates()
    f64b, f32b = jac.measure_fma_rates()
    f64, f32 = max(f64, f64b), max(f32, f32b)
    derived = 2.0 * sms * measured_peaks()[0].get("sm_max_mhz", 2070.0) * 1e6
    return {"fp64_gfma_s": round(f64 / 1e9, 1), "fp32_gfma_s": round(f32 / 1e9, 1),
            "fp64_tflops": round(2 * f64 / 1e12, 3), "fp64_fma_per_clk_per_sm_at_max_clock":
            round(f64 / (sms * measured_peaks()[0].get("sm_max_mhz", 2070.0) * 1e6), 3),
            "fp64_derived_gfma_s": round(derived / 1e9, 1),
            "how": "4 or 16 independent FMA chains per thread (recurrence or dot-product form), 4 or 8 blocks "
                   "of 256 threads per SM, CUDA events, best of all shapes over 2 calls"}


def composite_roofline(r, n, prec, peaks, dev, torch, fma=None):
    """Per-phase lower bound of the timed kernel: each FP64 pass (residual or sweep) is held by the larger of
    its HBM time and its FP64-FMA time (n^2 FMAs at the measured FP64 FMA rate, else 2 FP64 FMA per clock
    per SM), every other phase by its HBM time; the sum over the launch's phases against the measured
    kernel time."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if fma is not None:
        fp64_fma_s = fma["fp64_gfma_s"] * 1e9
        src = f"measured: {fma['fp64_gfma_s']:.0f} GFMA/s ({fma['fp64_tflops']:.2f} TFLOP/s, jacobi_measure_fma_rates)"
    else:
        fp64_fma_s = 2.0 * sms * peaks.get("sm_max_mhz", 2070.0) * 1e6
        src = (f"derived: 2 FP64 FMA/clock/SM x {sms} SMs x {peaks.get('sm_max_mhz', 2070.0):.0f} MHz = "
               f"{fp64_fma_s / 1e9:.0f} GFMA/s")
    hbm = peaks["hbm_gbs"] * 1e9
    es = ESIZE.get(prec.replace("+split", "").replace("+gs", ""), 8)
    per = {"sweep64": (8.0, True), "resid64": (8.0, True), "resid0": (0.0, False), "inner": (float(es), False),
           "narrow_inner": (8.0 + es, False)}
    total, rows = 0.0, {}
    for name, ph in r["phases"].items():
        if name not in per:
            continue
        bpe, fp64 = per[name]
        t_hbm = bpe * n * n / hbm
        t_fma = float(n) * n / fp64_fma_s if fp64 else 0.0
        t_min = max(t_hbm, t_fma)
        total += ph["count"] * t_min
        rows[name] = {"count": ph["count"], "bound": "fp64" if t_fma > t_hbm else "hbm", "min_us": round(t_min * 1e6, 1),
                      "measured_us": ph["mean_us"], "frac": round(t_min * 1e6 / ph["mean_us"], 3) if ph["mean_us"] else None}
    kernel_s = r["kernel_ms"] * 1e-3
    return {"min_ms": round(total * 1e3, 4), "kernel_ms": round(r["kernel_ms"], 4),
            "frac": round(total / kernel_s, 4) if kernel_s > 0 else None, "phases": rows,
            "fp64_fma_peak": src, "hbm_peak_gbs": peaks["hbm_gbs"]}


def phase_bandwidth(trace, n, prec):
    prec = prec.replace("+split", "").replace("+gs", "")
    """Per-phase-kind mean duration and algorithmic matrix bandwidth from the device-side trace of the
    last solve (each phase streams the whole matrix once: FP64 A, or the narrow copy)."""
    names = {0: ("sweep64", 8), 1: ("resid64", 8), 2: ("resid0", 0), 3: ("inner", ESIZE.get(prec, 8)),
             4: ("narrow_inner", 8 + ESIZE.get(prec, 8))}  # reads FP64 A, writes the narrow copy
    out = {}
    for kind, (name, es) in names.items():
        d = [(e - b) for k, b, e in trace if k == kind]
        if not d:
            continue
        # the first phase of a kind includes the kernel start-up; the mean over all is what is reported
        mean_ns = sum(d) / len(d)
        out[name] = {"count": len(d), "mean_us": round(mean_ns / 1e3, 2),
                     "gbs": round(es * float(n) * n / mean_ns, 1) if es and mean_ns > 0 else None}
    return out


def summarize(r, steps, n, prec):
    st = r["stats"]
    ms = r["ms_total"] / steps
    prec = prec.replace("+split", "").replace("+gs", "")
    es = ESIZE[prec]
    if prec == "fp64":
        bytes_launch = st["sweeps"] * 8.0 * n * n
    else:
        bytes_launch = max(st["outer_steps"] - 1, 0) * 8.0 * n * n + st["sweeps"] * es * float(n) * n
        if "narrow_inner" in r["phases"]:
            bytes_launch += 8.0 * n * n
    return {"solves_per_s": round(1e3 / ms, 3), "ms_per_solve": round(ms, 4), "kernel_ms": round(r["kernel_ms"], 4),
            "sweeps": st["sweeps"], "outer_steps": st["outer_steps"], "status": st["status"],
            "rel_residual": r["rel_residual_check"], "err_vs_xstar": r["err_vs_xstar"],
            "kernel_algorithmic_gbs": round(bytes_launch / (r["kernel_ms"] * 1e-3) / 1e9, 1),
            "phases": r["phases"],
            "gbs_per_sweep": round((8.0 if prec == "fp64" else es) * n * n / (r["kernel_ms"] * 1e-3 /
                                   max(st["sweeps"], 1)) / 1e9, 1) if prec == "fp64" else None}


def make_batch_inputs(count, seed, n_lo=64, n_hi=1024, f_lo=1.05, f_hi=2.0):
    """The batched workload: `count` dominant systems, n log-uniform in [n_lo, n_hi], f uniform in
    [f_lo, f_hi], generated on a thread pool."""
    import concurrent.futures as cf

    import synth
    ns, fs = synth.batch_shapes(count, n_lo, n_hi, f_lo, f_hi, seed)

    def one(k):
        A, B, _ = synth.dominant_system(int(ns[k]), float(fs[k]), synth.system_seed(seed, k))
        return A, B[:, 0].copy()

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        systems = list(ex.map(one, range(count)))
    return ns, fs, systems


def run_batch(args, jac, torch, dev):
    """4096 independent systems (n log-uniform in [64, 1024], f uniform in [1.05, 2.0]): one persistent
    work-queue kernel per solve, replayed from a CUDA graph, FP32 storage with FP64 refinement (FP64-FMA
    or split-float residuals) against the plain FP64 batched path, all to a 1e-10 relative residual;
    launch shapes from the autotuner."""
    import synth
    from paper_1403_5805_gb300 import autotune
    count = args.batch_count
    ns, fs, systems = make_batch_inputs(count, synth.BASE_SEED + 2)
    As = [torch.from_numpy(A).to(dev) for A, _ in systems]
    Bs = [torch.from_numpy(b).to(dev) for _, b in systems]
    sum_n2 = float(np.sum(ns.astype(np.float64) ** 2))
    stream = torch.cuda.current_stream(dev)
    out = {"count": count, "n_range": [64, 1024], "f_range": [1.05, 2.0], "sum_n2": sum_n2}
    for name in ("fp32_ir", "fp32_ir+split", "bf16_ir", "fp64"):
        prec, split = name.replace("+split", ""), name.endswith("+split")
        if args.batch_tuned:  # a fixed launch shape (profiler captures): rows per warp, CTAs per SM, inner tol
            rpw, cps, rt = args.batch_tuned.split(",")
            tuned = {"rows_per_warp": int(rpw), "ctas_per_sm": int(cps), "inner_rtol": 0.0 if prec == "fp64" else float(rt),
                     "cached": "fixed"}
        else:
            tuned = autotune.tune_batch(As, Bs, precision=prec, tol=TARGET, use_cache=True, split_residual=split)
        bs = jac.BatchSolver(As, Bs, precision=prec, rows_per_warp=tuned["rows_per_warp"],
                             ctas_per_sm=tuned["ctas_per_sm"], inner_rtol=tuned["inner_rtol"], split_residual=split)
        for _ in range(args.warmup):
            bs.solve_async(args.max_iter, TARGET)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        steps = args.batch_steps
        for _ in range(steps):
            bs.solve_async(args.max_iter, TARGET)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        st = bs.stats()
        ok = sum(1 for x in st if x.status == 0)
        sweeps = np.array([x.sweeps for x in st], dtype=np.float64)
        n2 = ns.astype(np.float64) ** 2
        if prec == "fp64":
            alg = float(np.sum(sweeps * 8.0 * n2))
            worst = float(max(x.final_delta for x in st))
        else:
            outer = np.array([x.outer_steps for x in st], dtype=np.float64)
            # setup pass (read A, write the narrow copy, the first inner sweep on the rounded values as
            # they are written) + FP64 residual passes + the other narrow inner sweeps
            es = 2.0 if prec == "bf16_ir" else 4.0
            alg = float(np.sum((8.0 + es) * n2 + np.maximum(outer - 1, 0) * 8.0 * n2
                               + np.maximum(sweeps - 1, 0) * es * n2))
            worst = float(max(x.rel_residual for x in st))
        out[name] = {"solves_per_s": round(count / (ms * 1e-3), 1), "ms_per_batch": round(ms, 4),
                     "converged": ok, "mean_sweeps": round(float(sweeps.mean()), 3),
                     "worst_rel_residual": worst, "algorithmic_gbs": round(alg / (ms * 1e-3) / 1e9, 1),
                     "grid": bs.grid, "tuned": {k: tuned[k] for k in ("rows_per_warp", "ctas_per_sm", "inner_rtol",
                                                                      "cached")}}
        if prec != "fp64":
            out[name]["mean_outer_steps"] = round(float(np.mean([x.outer_steps for x in st])), 3)
        bs.close()
    out["mixed_vs_fp64_solves_ratio"] = round(out["fp32_ir"]["solves_per_s"] / out["fp64"]["solves_per_s"], 3)
    out["mixed_split_vs_fp64_solves_ratio"] = round(
        out["fp32_ir+split"]["solves_per_s"] / out["fp64"]["solves_per_s"], 3)
    out["bf16_vs_fp64_solves_ratio"] = round(out["bf16_ir"]["solves_per_s"] / out["fp64"]["solves_per_s"], 3)
    return out


def run_sparse(args, jac, torch, dev):
    """PDE-shaped sparse workload: the 5-point stencil of a variable-coefficient diffusion operator on an
    N x N grid (N = --sparse-grid, 4.19 M unknowns by default), f = 1.05 (rho(T) <= 1/1.05), kept in the
    format setup picks (DIA: the stencil's 4 diagonals, no column array).  Times a fixed count of sweeps
    (per-sweep HBM rate against the measured copy rate) and a full solve to max|dx| < 1e-12, and the CPU
    oracle on a few sweeps."""
    import synth
    N = args.sparse_grid
    rp, ci, v, B, Xs = synth.stencil_system((N, N), 1.05, seed=synth.BASE_SEED + 6)
    n = B.shape[0]
    nnz_off = int(rp[-1]) - n
    stream = torch.cuda.current_stream(dev)
    t_rp, t_ci, t_v, t_b = (torch.from_numpy(a).to(dev) for a in (rp, ci, v, B[:, 0].copy()))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    fl = jac.binding.FLAG_CSR_ELL if args.sparse_ell else 0  # --sparse-ell: keep sliced ELL
    s = jac.CsrSolver(t_rp, t_ci, t_v, t_b, flags=fl)
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    setup_ms = ev[0].elapsed_time(ev[1])
    info = s.info()
    out = torch.empty(n, dtype=torch.float64, device=dev)

    def timed(max_iter, tol, reps):
        for _ in range(2):
            s.solve_async(None, max_iter, tol, out)
        torch.cuda.synchronize(dev)
        ev[0].record(stream)
        for _ in range(reps):
            s.solve_async(None, max_iter, tol, out)
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        return ev[0].elapsed_time(ev[1]) / reps, s.last_stats()

    K = args.sparse_sweeps
    ms_fixed, st_fixed = timed(K, 1e-300, 3)
    tr = s.trace()
    per = sorted(b - a for a, b in tr[1:])  # the first sweep also holds the launch
    sweep_us = per[len(per) // 2] / 1e3
    # T values (+ int32 columns in sliced ELL; DIA has none), C, x read, x written
    alg_bytes = (8.0 if info["format"] == "dia" else 12.0) * nnz_off + 24.0 * n
    peaks, kind = measured_peaks()
    gbs = alg_bytes / (sweep_us * 1e-6) / 1e9
    ms_solve, st = timed(5000, 1e-12, 3)
    err = float((out - torch.from_numpy(Xs[:, 0]).to(dev)).abs().max().item())
    s.close()
    # the same stopping quantity as the refined solves: ||b - A x|| / ||b|| < 1e-10 (of the previous iterate)
    s = jac.CsrSolver(t_rp, t_ci, t_v, t_b, norm="resid", flags=fl)
    ms_resid, st_resid = timed(5000, 1e-10, 3)
    import oracle
    refined = {}
    for prec in ("bf16_ir", "fp32_ir"):  # the same system, mixed precision, to ||b - A x|| / ||b|| <= 1e-10
        r = jac.CsrSolver(t_rp, t_ci, t_v, t_b, precision=prec, flags=fl)
        for _ in range(2):
            r.solve_async(None, 1, 1e-10, out)
        torch.cuda.synchronize(dev)
        ev[0].record(stream)
        for _ in range(3):
            r.solve_async(None, 1, 1e-10, out)
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        rst = r.last_stats()
        ms_r = ev[0].elapsed_time(ev[1]) / 3
        inner = [b - a for (a, b), k in zip(r.trace(), r.kinds()) if k == 3][1:]
        refined[prec] = {"ms": round(ms_r, 3), "solves_per_s": round(1e3 / ms_r, 3), "status": int(rst.status),
                         "inner_sweeps": int(rst.sweeps), "outer_steps": int(rst.outer_steps),
                         "rel_residual_checked": oracle.csr_residual(rp, ci, v, B, out.cpu().numpy())[1],
                         "median_inner_sweep_us": round(sorted(inner)[len(inner) // 2] / 1e3, 2) if inner else None,
                         "vs_fp64_same_target": round(ms_resid / ms_r, 2)}
        r.close()
    import time as _t
    k_cpu = 3
    t0 = _t.perf_counter()
    oracle.csr_jacobi(rp, ci, v, B, max_iter=k_cpu, tol=1e-300)
    cpu_ms_sweep = (_t.perf_counter() - t0) * 1e3 / k_cpu
    s.close()
    return {"workload": f"2-D 5-point variable-coefficient diffusion stencil, {N} x {N} grid, f = 1.05, "
                        f"planted solution; "
                        + (f"DIA ({info['diagonals']} diagonals, 32-row slices)" if info["format"] == "dia"
                           else "sliced ELL (32-row slices)"),
            "format": info["format"],
            "n": n, "nnz": int(rp[-1]), "stored_slots": info["stored_slots"], "grid": info["grid"],
            "setup_ms": round(setup_ms, 3),
            "sweeps": {"count": int(st_fixed.sweeps), "ms_total": round(ms_fixed, 4),
                       "median_sweep_us": round(sweep_us, 2), "algorithmic_bytes_per_sweep": alg_bytes,
                       "achieved_gbs": round(gbs, 1), "peak_gbs": peaks["hbm_gbs"],
                       "frac": round(gbs / peaks["hbm_gbs"], 4),
                       "peak_source": f"{kind} (MEASURED_PEAKS.json hbm_gbs)"},
            "solve": {"tol": 1e-12, "status": int(st.status), "sweeps": int(st.sweeps), "ms": round(ms_solve, 3),
                      "solves_per_s": round(1e3 / ms_solve, 3), "err_vs_xstar": err},
            "solve_resid": {"tol": 1e-10, "norm": "relative residual", "status": int(st_resid.status),
                            "sweeps": int(st_resid.sweeps), "ms": round(ms_resid, 3),
                            "solves_per_s": round(1e3 / ms_resid, 3)},
            "refined": refined,
            "cpu_oracle": {"ms_per_sweep": round(cpu_ms_sweep, 1), "cores": 1,
                           "sample": f"{k_cpu} sweeps of the full system, one thread"},
            "gpu_vs_cpu_sweep_ratio": round(cpu_ms_sweep * 1e3 / sweep_us, 1)}


def run_many_rhs(args, jac, torch, dev):
    """n = 32768 with 64 right-hand sides, f = 1.1: BF16 sweeps on tcgen05 tensor cores with FP64
    refinement against the plain FP64 path (each sweep a dense FP64 pass), both to 1e-10."""
    import synth
    n, r = args.mrhs_n, 64
    A, B, Xs = synth.dominant_system(n, 1.1, seed=synth.BASE_SEED + 3, nrhs=r)
    At = torch.from_numpy(A).to(dev)
    del A
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).to(dev)
    Xst = torch.from_numpy(np.ascontiguousarray(Xs.T)).to(dev)
    stream = torch.cuda.current_stream(dev)
    out = {"n": n, "nrhs": r, "dominance": 1.1}
    for prec, steps in (("bf16_ir+tc", args.mrhs_steps), ("bf16_ir", args.mrhs_steps),
                        ("bf16_ir+split", args.mrhs_steps), ("fp64", 1)):
        torch.cuda.synchronize(dev)
        t_setup = time.perf_counter()
        solver = jac.MultiSolver(At, Bt, precision=prec.split("+")[0], split_residual=prec.endswith("+split"),
                                 tc_residual=prec.endswith("+tc"))
        torch.cuda.synchronize(dev)
        setup_ms = (time.perf_counter() - t_setup) * 1e3
        X, st = solver.solve(max_iter=5000, tol=TARGET if prec != "fp64" else args.fp64_tol)  # warm-up
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            X, st = solver.solve(max_iter=5000, tol=TARGET if prec != "fp64" else args.fp64_tol, out=X)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        err = (X - Xst).abs().amax(dim=1)
        phases = {}
        rname = ("resid64_split_fp32" if prec.endswith("+split") else
                 "resid64_tc_digits" if prec.endswith("+tc") else "resid64_fp64")
        for kind, name, es, flop in ((3, "inner_tcgen05_bf16", 2, True), (1, rname, 8, True),
                                     (0, "sweep64_fp64", 8, True)):
            d = [(e - b) for k, b, e in solver.trace() if k == kind]
            if d:
                mean = sum(d) / len(d)
                phases[name] = {"count": len(d), "mean_us": round(mean / 1e3, 1),
                                "matrix_gbs": round(es * float(n) * n / mean, 1),
                                "tflops": round(2.0 * n * n * r / mean / 1e3, 2)}
        out[prec] = {"solves_per_s": round(1e3 / ms, 3), "ms_per_solve": round(ms, 2), "setup_ms": round(setup_ms, 1),
                     "status": st.status,
                     "sweeps": st.sweeps, "outer_steps": st.outer_steps, "rel_residual": st.rel_residual,
                     "max_err_vs_xstar_per_rhs": float(err.max().item()), "phases": phases}
        solver.close()
    out["mixed_vs_fp64_solves_ratio"] = round(out["bf16_ir"]["solves_per_s"] / out["fp64"]["solves_per_s"], 3)
    out["mixed_tc_vs_fp64_solves_ratio"] = round(out["bf16_ir+tc"]["solves_per_s"] / out["fp64"]["solves_per_s"], 3)
    out["mixed_split_vs_fp64_solves_ratio"] = round(
        out["bf16_ir+split"]["solves_per_s"] / out["fp64"]["solves_per_s"], 3)
    return out


def run_symmetric(args, jac, torch, dev):
    """A symmetric n = 16384 system (the dominant generator mirrored about the diagonal, f = 1.05), BF16 and
    FP32 inner sweeps with FP64 refinement to a 1e-10 relative residual: the narrow copy in full (the
    persistent single-system kernel) against the packed upper tiles of JACOBI_FLAG_SYMMETRIC (half the bytes
    of every inner sweep).  Per inner sweep: the mean phase time of the trace (kernel time between CUDA
    events for the packed form: its tile launch and its finish launch) and the bytes of the narrow copy it
    reads."""
    import synth
    n = args.sym_n
    A, B, Xs = synth.symmetric_system(n, 1.05, seed=synth.BASE_SEED + 7)
    At = torch.from_numpy(A).to(dev)
    bt = torch.from_numpy(B[:, 0].copy()).to(dev)
    out = {"n": n, "dominance": 1.05}
    for prec, es in (("bf16_ir", 2), ("fp32_ir", 4)):
        for sym in (False, True):
            name = prec + ("+sym" if sym else "")
            s = jac.DeviceSolver(At, bt, precision=prec, symmetric=sym)
            X, st = s.solve(max_iter=5000, tol=TARGET)  # warm-up (and the fused narrow copy)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            reps = 5
            for _ in range(reps):
                X, st = s.solve(max_iter=5000, tol=TARGET, out=X)
            torch.cuda.synchronize(dev)
            ms = (time.perf_counter() - t0) * 1e3 / reps
            tr = s.trace()
            inner = [(e - b) for k, b, e in tr if k == 3]
            resid = [(e - b) for k, b, e in tr if k == 1]
            mean_inner = sum(inner) / len(inner) if inner else None
            stored = (n * n / 2.0 + 64.0 * n) if sym else float(n) * n   # entries of the narrow copy read per sweep
            out[name] = {"ms_per_solve": round(ms, 3), "status": st.status, "inner_sweeps": st.sweeps,
                         "outer_steps": st.outer_steps, "rel_residual": st.rel_residual,
                         "err_vs_xstar": float((X - torch.from_numpy(Xs[:, 0].copy()).to(dev)).abs().max().item()),
                         "inner_sweep_us": round(mean_inner / 1e3, 2) if mean_inner else None,
                         "inner_sweep_gbs": round(es * stored / mean_inner, 1) if mean_inner else None,
                         "resid64_us": round(sum(resid) / len(resid) / 1e3, 1) if resid else None}
            s.close()
        full, half = out[prec]["inner_sweep_us"], out[prec + "+sym"]["inner_sweep_us"]
        out[prec + "_inner_sweep_speedup"] = round(full / half, 3) if full and half else None
    return out


def run_serve(args, jac, torch, dev, seconds, other_seconds=None):
    """Poisson arrivals at 2000 requests/s (n log-uniform in [256, 8192], r uniform in {1..16}, f uniform
    in [1.05, 1.5], FP64 inputs generated on the device at admission), served with continuous batching
    under a 100 GB budget to a 1e-10 relative residual: with residual rounds on the tensor cores (the
    FP64-accurate digit split) for `seconds` of arrivals, and with FP64-FMA and split-float residual
    rounds for `other_seconds` (default: the same); latency from each request's scheduled arrival to the
    moment its result is polled.  Beside them, the same trace's first `serve_fp64_seconds` solved one
    request at a time by the plain FP64 path."""
    import time as _time

    import synth
    rate = 2000.0
    other_seconds = seconds if other_seconds is None else other_seconds
    traces = {}

    def trace(sec):
        if sec not in traces:
            traces[sec] = synth.serving_trace(rate, sec, seed=synth.BASE_SEED + 4)
        return traces[sec]

    free, _ = torch.cuda.mem_get_info(dev)
    budget = int(min(args.serve_budget_gb * 1e9, free - 8e9))

    def served(mode):
        t, ns, rs, fs, seeds = trace(seconds if mode == "tc" else other_seconds)
        srv = jac.Server(budget_bytes=budget, split_residual=mode == "split", tc_residual=mode == "tc",
                         inner_rtol=args.serve_inner_rtol)
        outs, arrive, lat, stats = {}, {}, {}, {}
        k = 0
        total = len(t)
        active_samples = []
        t0 = _time.perf_counter()
        while len(lat) < total:
            now = _time.perf_counter() - t0
            while k < total and t[k] <= now:
                out = torch.empty(int(rs[k]), int(ns[k]), dtype=torch.float64, device=dev)
                rid = srv.submit_generated(int(ns[k]), int(rs[k]), float(fs[k]), int(seeds[k]), out)
                outs[rid] = (k, out)
                arrive[rid] = t[k]
                k += 1
            active, pending = srv.step()
            active_samples.append(active + pending)
            done_t = _time.perf_counter() - t0
            for rid, st in srv.poll():
                lat[rid] = done_t - arrive[rid]
                stats[rid] = (st.status, st.rel_residual, st.outer_steps, st.sweeps)
                kk, out = outs[rid]
                if kk % max(1, total // 16) == 0:  # keep a sample for the host-side check
                    outs[rid] = (kk, out)
                else:
                    del outs[rid]
            if k >= total and active == 0 and pending == 0 and len(lat) < total:
                for rid, st in srv.poll():
                    lat[rid] = _time.perf_counter() - t0 - arrive[rid]
        wall = _time.perf_counter() - t0
        rounds = srv.rounds()
        srv.close()
        L = np.array(sorted(lat.values())) * 1e3
        ok = sum(1 for v in stats.values() if v[0] == 0)
        worst = max(v[1] for v in stats.values())
        # host check of sampled results (inputs regenerated from their seeds)
        checked = []
        for rid, (kk, out) in list(outs.items())[:8]:
            A, B = synth.serving_request(int(ns[kk]), int(rs[kk]), float(fs[kk]), int(seeds[kk]))
            X = out.cpu().numpy().T
            R = B - A @ X
            checked.append(float(np.max(np.abs(R).max(axis=0) / np.abs(B).max(axis=0))))
        return {"offered_rate": rate, "seconds": seconds, "requests": total, "converged": ok,
                "throughput_per_s": round(total / wall, 1), "wall_s": round(wall, 3),
                "p50_ms": round(float(np.percentile(L, 50)), 3), "p99_ms": round(float(np.percentile(L, 99)), 3),
                "max_ms": round(float(L[-1]), 3), "rounds": rounds, "arrival_window_s": seconds if mode == "tc" else other_seconds,
                "mean_in_system": round(float(np.mean(active_samples)), 1),
                "mean_outer_steps": round(float(np.mean([v[2] for v in stats.values()])), 2),
                "mean_inner_sweeps": round(float(np.mean([v[3] for v in stats.values()])), 2),
                "worst_rel_residual": worst, "sampled_host_residuals_max": max(checked) if checked else None,
                "budget_gb": round(budget / 1e9, 1),
                "residual": {"split": "split-float (FP32 units)", "fp64": "FP64 FMAs",
                             "tc": "tensor cores, BF16 digit split (FP64-accurate)"}[mode]}

    modes = args.serve_modes.split(",")
    served_tc = served("tc") if "tc" in modes else None
    served_fp64_resid = served("fp64") if "fp64" in modes else None
    served_split = served("split") if "split" in modes else None

    # the plain FP64 path, one request at a time, on the first seconds of the same trace
    t, ns, rs, fs, seeds = trace(seconds)
    m = int(np.searchsorted(t, args.serve_fp64_seconds))
    lat64 = []
    t0 = _time.perf_counter()
    for q in range(m):
        now = _time.perf_counter() - t0
        if t[q] > now:
            _time.sleep(t[q] - now)
        n, r = int(ns[q]), int(rs[q])
        A, Bc = jac.generate_request(n, r, float(fs[q]), int(seeds[q]), device=dev)
        if r == 1:
            sol = jac.DeviceSolver(A, Bc.reshape(-1), precision="fp64", norm="resid")
            X, st = sol.solve(max_iter=5000, tol=TARGET)
        else:
            sol = jac.MultiSolver(A, Bc, precision="fp64", norm="resid")
            X, st = sol.solve(max_iter=5000, tol=TARGET)
        sol.close()
        lat64.append(_time.perf_counter() - t0 - t[q])
    wall64 = _time.perf_counter() - t0
    L64 = np.array(sorted(lat64)) * 1e3
    fp64 = {"requests": m, "arrival_window_s": args.serve_fp64_seconds,
            "throughput_per_s": round(m / wall64, 1) if m else None,
            "p50_ms": round(float(np.percentile(L64, 50)), 3) if m else None,
            "p99_ms": round(float(np.percentile(L64, 99)), 3) if m else None}
    ratio = (lambda a: round(a["throughput_per_s"] / fp64["throughput_per_s"], 2)
             if (a and fp64["throughput_per_s"]) else None)
    return {"served_fp32_ir_tc_residual": served_tc, "served_fp32_ir": served_fp64_resid,
            "served_fp32_ir_split_residual": served_split,
            "one_at_a_time_fp64": fp64, "throughput_ratio_tc_residual": ratio(served_tc),
            "throughput_ratio": ratio(served_fp64_resid), "throughput_ratio_split_residual": ratio(served_split)}


def run_hard(args, jac, torch, dev, ws):
    """The same n = 16384 solve on the paper-shaped generator (off-diagonals uniform [0, 1), positive
    diagonal f * row sum, f = 1.05: rho(T) = 1/f exactly, so plain Jacobi needs hundreds of sweeps)."""
    import synth
    n = args.n
    A, B, Xs = synth.hard_system(n, 1.05, seed=synth.BASE_SEED + 5)
    At = torch.from_numpy(A).to(dev)
    Bt = torch.from_numpy(B[:, 0].copy()).to(dev)
    del A
    stream = torch.cuda.current_stream(dev)
    out = torch.empty(n, dtype=torch.float64, device=dev)
    res = {"n": n, "dominance": 1.05, "rho_T": round(1 / 1.05, 6)}
    # Gauss-Seidel stops on the max-norm change (its change is not the residual); 1e-11 lands below the
    # 1e-10 relative residual, which is measured and reported
    for name, prec, tol, norm, method in (("bf16_ir", "bf16_ir", TARGET, "inf", "jacobi"),
                                          ("fp32_ir", "fp32_ir", TARGET, "inf", "jacobi"),
                                          ("fp64", "fp64", TARGET, "resid", "jacobi"),
                                          ("fp64_gauss_seidel", "fp64", 1e-11, "inf", "sor")):
        s = jac.DeviceSolver(At, Bt, precision=prec, norm=norm, workspace=ws, method=method)
        s.solve_async(None, 20000, tol, out)  # warm-up
        torch.cuda.synchronize(dev)
        steps = 1 if name == "fp64" else 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            s = jac.DeviceSolver(At, Bt, precision=prec, norm=norm, workspace=ws, method=method)
            s.solve_async(None, 20000, tol, out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        st = s.last_stats()
        res[name] = {"solves_per_s": round(1e3 / ms, 3), "ms_per_solve": round(ms, 2), "status": st.status,
                     "sweeps": st.sweeps, "outer_steps": st.outer_steps, "rel_residual": s.residual(out)}
    res["bf16_vs_fp64_solves_ratio"] = round(res["bf16_ir"]["solves_per_s"] / res["fp64"]["solves_per_s"], 2)
    res["gauss_seidel_vs_fp64_solves_ratio"] = round(
        res["fp64_gauss_seidel"]["solves_per_s"] / res["fp64"]["solves_per_s"], 2)
    return res


def run_small(args, jac, torch, dev):
    """The small system n = 512 (f = 1.25, tol 1e-12 on max|dx|), on the dominant generator (rho(T) small:
    ~10 sweeps) and the paper-shaped one (rho(T) = 0.8: ~110 sweeps).  A is 2.1 MB and stays in L2, so a
    sweep is bound by the grid barrier and the FP64 rate, not HBM: per-sweep time from the device trace,
    the solve with and without setup, and the rate at which the L2-resident A is swept, for the default
    grid and smaller ones."""
    import synth
    n, f = 512, 1.25
    stream = torch.cuda.current_stream(dev)
    out = torch.empty(n, dtype=torch.float64, device=dev)
    res = {"n": n, "dominance": f, "tol": 1e-12, "a_bytes": 8 * n * n}
    for gen_name, gen, seed in (("dominant", synth.dominant_system, synth.BASE_SEED),
                                ("paper_shaped", synth.hard_system, synth.BASE_SEED + 7)):
        A, B, Xs = gen(n, f, seed=seed)
        At = torch.from_numpy(A).to(dev)
        Bt = torch.from_numpy(B[:, 0].copy()).to(dev)
        rows = {}
        for grid in (0, 16, 38, 76):
            s = jac.DeviceSolver(At, Bt, precision="fp64", grid=grid)
            for _ in range(3):
                s.solve_async(None, 2000, 1e-12, out)
            torch.cuda.synchronize(dev)
            reps = 50
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                s.solve_async(None, 2000, 1e-12, out)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            solve_us = e0.elapsed_time(e1) * 1e3 / reps
            st = s.last_stats()
            tr = [(e - b) for k, b, e in s.trace() if k == 0]
            sweep_us = (sorted(tr)[len(tr) // 2] / 1e3) if tr else None
            t0 = time.perf_counter()
            for _ in range(reps):  # setup + solve through the public API, each waited for
                s2 = jac.DeviceSolver(At, Bt, precision="fp64", grid=grid)
                s2.solve_async(None, 2000, 1e-12, out)
                s2.last_stats()
            with_setup_us = (time.perf_counter() - t0) * 1e6 / reps
            rows["auto" if grid == 0 else str(grid)] = {
                "status": st.status, "sweeps": st.sweeps, "solve_us": round(solve_us, 2),
                "median_sweep_us": round(sweep_us, 3) if sweep_us else None,
                "l2_sweep_gbs": round(8.0 * n * n / (sweep_us * 1e3), 1) if sweep_us else None,
                "solves_per_s": round(1e6 / solve_us, 1), "setup_and_solve_us": round(with_setup_us, 1),
                "err_vs_xstar": float((out - torch.from_numpy(Xs[:, 0].copy()).to(dev)).abs().max().item())}
        res[gen_name] = rows
    return res


def run_e2e(args, jac, torch, dev, A, B, ws):
    """Same metric through the public API from pinned host buffers: per step the H2D of A and B, setup,
    solve and the D2H read of X, all inside the timed region.  Two solvers alternate on two CUDA streams
    (two workspaces), so one step's host-to-device copy (copy engine) overlaps the previous step's
    setup kernels and solve, as an application streaming independent systems would run them; the
    sequential form (one stream, each step waited for) is reported beside it."""
    n = args.n
    Ah = torch.from_numpy(A).pin_memory()
    Bh = torch.from_numpy(B[:, 0].copy()).pin_memory()
    streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    wss = [ws, torch.empty_like(ws)]
    outs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(2)]
    Xhs = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(2)]
    steps = max(1, min(args.steps, args.e2e_steps))

    def launch(k):
        q = k % 2
        with torch.cuda.stream(streams[q]):
            s = jac.DeviceSolver(Ah, Bh, precision=args.precision, workspace=wss[q], device=dev,
                                 inner_rtol=args.inner_rtol, max_inner=args.max_inner, stream=streams[q])
            s.solve_async(None, args.max_iter, TARGET, outs[q])
            Xhs[q].copy_(outs[q], non_blocking=True)
        return s

    def run(count, pipelined):
        pending, st = None, None
        for k in range(count):
            s = launch(k if pipelined else 0)
            if not pipelined:
                st = s.last_stats()  # waits for the stream: X has landed in host memory
                continue
            if pending is not None:
                st = pending.last_stats()  # the previous step, overlapped with this one's copy
            pending = s
        if pending is not None:
            st = pending.last_stats()
        return st

    # the host link is shared with the machine's other tenants and its rate swings between runs, so each
    # form is timed in three blocks of `steps` solves and the median block is reported, all blocks beside
    out, blocks = {}, {}
    for name, pipelined in (("pipelined", True), ("sequential", False)):
        run(max(2, args.warmup), pipelined)
        torch.cuda.synchronize(dev)
        rates = []
        for _ in range(3):
            t0 = time.perf_counter()
            st = run(steps, pipelined)
            torch.cuda.synchronize(dev)
            sec = (time.perf_counter() - t0) / steps
            rates.append(round(1.0 / sec, 3) if st.status == 0 else 0.0)
        blocks[name] = rates
        out[name] = sorted(rates)[1]
    return {"value": out["pipelined"], "unit": "solves/s", "steps": 3 * steps,
            "h2d_bytes_per_step": int(8 * n * n + 8 * n), "d2h_bytes_per_step": int(8 * n),
            "sequential_value": out["sequential"], "blocks_solves_per_s": blocks,
            "path": "host pinned A,B -> jacobi_setup_ex (H2D copy into the workspace) -> jacobi_solve_async -> "
                    "X to pinned host; two solvers on two streams, each step's H2D overlapping the previous "
                    "step's solve"}


# --------------------------------------------------------------------------------- CPU oracle

def oracle_solve(A, B, threads):
    import oracle
    # FP64 Jacobi with the relative-residual stop (previous iterate), the same 1e-10 target
    return oracle.jacobi(A, B, max_iter=2000, tol=TARGET, norm=oracle.NORM_RESID, nthreads=threads)


def cpu_baseline(A, B, n, budget_s: float = 12.0):
    import oracle
    threads = os.cpu_count() or 1
    oracle.build()
    t0 = time.perf_counter()
    solves = 0
    res = None
    while True:
        res = oracle_solve(A, B, threads)
        solves += 1
        if time.perf_counter() - t0 >= budget_s or solves >= 5:
            break
    sec = (time.perf_counter() - t0) / solves
    # and the plain serial loop: two sweeps of the same system on one core
    t1 = time.perf_counter()
    oracle.jacobi(A, B, max_iter=2, tol=1e-300, nthreads=1)
    single_ms = (time.perf_counter() - t1) * 1e3 / 2
    return {"value": round(1.0 / sec, 4), "unit": "solves/s", "cores": threads, "kind": "oracle",
            "sample": f"{solves} full FP64 oracle solve(s) of the n={n} system (OpenMP rows, "
                      f"{res.iters} sweeps each, relative-residual stop 1e-10)",
            "single_core_ms_per_sweep": round(single_ms, 1)}, res.X[:, 0].copy()


def run_reference(args, world, rank):
    """Reference arm: the plain FP64 CPU oracle on the machine's host cores (rank 0 only)."""
    import numpy as np  # noqa: F401

    import synth
    if rank != 0:
        return None
    n, f = args.n, args.f
    A, B, _ = synth.dominant_system(n, f, seed=synth.BASE_SEED + 1)
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    for _ in range(max(0, min(args.warmup, 1))):
        oracle_solve(A, B, threads)
    t0 = time.perf_counter()
    res = None
    for _ in range(args.steps):
        res = oracle_solve(A, B, threads)
    sec = (time.perf_counter() - t0) / args.steps
    value = 1.0 / sec
    return {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Philox4x32-10)",
            "config": {"workload": f"single dense system n={n}, f={f}, 1 RHS, FP64 Jacobi (CPU oracle) to "
                                   f"rel. residual 1e-10", "n": n, "dominance": f},
            "cpu_baseline": {"value": round(value, 4), "unit": "solves/s", "cores": threads, "kind": "oracle",
                             "sample": f"{args.steps} full oracle solves, {res.iters} sweeps each"},
            "e2e": {"value": round(value, 4), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--f", type=float, default=1.05)
    ap.add_argument("--precision", default="bf16_ir", choices=list(ESIZE) + ["fp64+gs"],
                    help="the timed path; fp64+gs is the chained Gauss-Seidel solve")
    ap.add_argument("--fp64-tol", type=float, default=1e-12, dest="fp64_tol",
                    help="stopping threshold of the plain FP64 path (max-norm change)")
    ap.add_argument("--max-iter", type=int, default=5000, dest="max_iter")
    ap.add_argument("--e2e-steps", type=int, default=10, dest="e2e_steps")
    ap.add_argument("--inner-rtol", type=float, default=0.0, dest="inner_rtol",
                    help="mixed paths: inner-sweep stop (relative change); 0 = library default")
    ap.add_argument("--max-inner", type=int, default=0, dest="max_inner")
    ap.add_argument("--split-residual", action="store_true", dest="split_residual",
                    help="mixed paths: FP64-accurate residual on the FP32 units (split-float)")
    ap.add_argument("--quick", action="store_true", help="skip the comparison paths")
    ap.add_argument("--no-cpu-baseline", action="store_true", dest="no_cpu_baseline")
    ap.add_argument("--no-e2e", action="store_true", dest="no_e2e")
    ap.add_argument("--no-batch", action="store_true", dest="no_batch")
    ap.add_argument("--no-mrhs", action="store_true", dest="no_mrhs")
    ap.add_argument("--no-serve", action="store_true", dest="no_serve")
    ap.add_argument("--no-hard", action="store_true", dest="no_hard")
    ap.add_argument("--no-small", action="store_true", dest="no_small")
    ap.add_argument("--no-sparse", action="store_true", dest="no_sparse")
    ap.add_argument("--sparse-grid", type=int, default=2048, dest="sparse_grid",
                    help="side of the 2-D stencil grid of the sparse section")
    ap.add_argument("--sparse-sweeps", type=int, default=200, dest="sparse_sweeps")
    ap.add_argument("--sparse-ell", action="store_true", dest="sparse_ell",
                    help="keep the sparse section's matrix in sliced ELL instead of the DIA form setup picks")
    ap.add_argument("--serve-seconds", type=float, default=60.0, dest="serve_seconds",
                    help="arrival window of the tensor-core-residual server (the serving configuration's 60 s)")
    ap.add_argument("--serve-window", type=float, default=5.0, dest="serve_window",
                    help="arrival window of the FP64-FMA and split-float servers in the default run")
    ap.add_argument("--serve-budget-gb", type=float, default=100.0, dest="serve_budget_gb",
                    help="device-memory budget of the serving arena (the configuration's 100 GB; a few GB "
                         "for a profiler capture)")
    ap.add_argument("--serve-inner-rtol", type=float, default=0.0, dest="serve_inner_rtol",
                    help="serving: inner-sweep stop (relative change); 0 = library default")
    ap.add_argument("--serve-modes", default="tc,fp64,split", dest="serve_modes",
                    help="serving: which residual forms to run (fp64, split)")
    ap.add_argument("--serve-fp64-seconds", type=float, default=1.0, dest="serve_fp64_seconds")
    ap.add_argument("--sym-n", type=int, default=16384, dest="sym_n")
    ap.add_argument("--only", choices=["batch", "mrhs", "serve", "sparse", "small", "sym"], default=None,
                    help="run one secondary workload alone (profiling)")
    ap.add_argument("--batch-tuned", default="", dest="batch_tuned",
                    help="batched section: fixed 'rows_per_warp,ctas_per_sm,inner_rtol' instead of the autotuner")
    ap.add_argument("--mrhs-n", type=int, default=32768, dest="mrhs_n")
    ap.add_argument("--mrhs-steps", type=int, default=3, dest="mrhs_steps")
    ap.add_argument("--batch-count", type=int, default=4096, dest="batch_count")
    ap.add_argument("--batch-steps", type=int, default=10, dest="batch_steps")
    args = ap.parse_args()
    world, rank, local = dist_env()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        if world > 1 and rank != 0:
            return
        res = run_reference(args, world, rank)
        print(json.dumps(res), flush=True)
        return
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    res = run_ours(args, world, rank, local)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
