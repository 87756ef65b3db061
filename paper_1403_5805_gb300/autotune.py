"""Autotuner for the launch shapes and inner tolerances of the solver kernels.

It times candidate configurations of a concrete workload through the C ABI (CUDA events on the
solver's stream, after a warm-up solve) and keeps the fastest one whose every system converged.
Results are cached in a JSON file keyed by the workload signature (device name, precision, system
count and a histogram of the sizes), so a workload is tuned once per machine.

Tuned knobs
  batch:  rows per warp (1, 2, 4, 8), resident CTAs per SM (all that fit, 4 with the register-limited
          build, 2, 1) and, for the mixed
          precisions, the inner-sweep stopping tolerance.
  single: the inner-sweep stopping tolerance of the mixed precisions.
"""
from __future__ import annotations

import hashlib
import json
import os
import threading

import numpy as np

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("JACOBI_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "jacobi_gb300", "tune.json"))


def _load_cache() -> dict:
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(key: str, value: dict) -> None:
    with _lock:
        data = _load_cache()
        data[key] = value
        path = cache_path()
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)


def _signature(kind: str, precision: str, sizes) -> str:
    import torch
    sizes = np.asarray(sizes, dtype=np.int64)
    hist = np.histogram(np.log2(np.maximum(sizes, 1)), bins=16, range=(0, 16))[0]
    h = hashlib.sha256(hist.tobytes() + str(len(sizes)).encode()).hexdigest()[:16]
    return f"{kind}|{torch.cuda.get_device_name()}|{precision}|{len(sizes)}|{h}"


def _time(fn, reps: int) -> float:
    import torch
    fn()  # warm-up (also captures the batch graph)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_batch(As, Bs, precision: str = "fp32_ir", max_iter: int = 5000, tol: float = 1e-10, reps: int = 3,
               use_cache: bool = True, workspace=None, split_residual: bool = False) -> dict:
    """Best ``{rows_per_warp, ctas_per_sm, inner_rtol, ms}`` for this batch."""
    from .binding import BatchSolver
    key = _signature("batch", precision + ("+split" if split_residual else ""), [a.shape[0] for a in As])
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return dict(hit, cached=True)
    rtols = [0.0] if precision == "fp64" else [2.0 ** -10, 2.0 ** -14, 2.0 ** -18]
    best = None
    trials = []
    for rpw in (1, 2, 4, 8):
        for cps in (0, 4, 2, 1):
            for rt in rtols:
                bs = BatchSolver(As, Bs, precision=precision, rows_per_warp=rpw, ctas_per_sm=cps, inner_rtol=rt,
                                 workspace=workspace, split_residual=split_residual)
                workspace = bs.workspace
                ms = _time(lambda: bs.solve_async(max_iter, tol), reps)
                ok = all(s.status == 0 for s in bs.stats())
                grid = bs.grid
                bs.close()
                trials.append({"rows_per_warp": rpw, "ctas_per_sm": cps, "inner_rtol": rt, "ms": ms, "ok": ok,
                               "grid": grid})
                if ok and (best is None or ms < best["ms"]):
                    best = trials[-1]
    if best is None:
        raise RuntimeError("no batch configuration converged")
    result = dict(best, trials=len(trials))
    if use_cache:
        _store(key, result)
    return dict(result, cached=False)


def tune_single(A, B, precision: str, max_iter: int = 5000, tol: float = 1e-10, reps: int = 5,
                use_cache: bool = True) -> dict:
    """Best inner-sweep tolerance ``{inner_rtol, ms}`` of a mixed-precision single-system solve."""
    from .binding import DeviceSolver
    key = _signature("single", precision, [A.shape[0]])
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return dict(hit, cached=True)
    best = None
    ws = None
    for rt in (2.0 ** -8, 2.0 ** -10, 2.0 ** -12, 2.0 ** -14, 2.0 ** -16, 2.0 ** -20):
        def run():
            nonlocal ws
            s = DeviceSolver(A, B, precision=precision, inner_rtol=rt, workspace=ws)
            ws = s.workspace
            s.solve_async(None, max_iter, tol)
            return s
        ms = _time(run, reps)
        st = run().last_stats()
        if st.status == 0 and (best is None or ms < best["ms"]):
            best = {"inner_rtol": rt, "ms": ms, "outer_steps": st.outer_steps, "sweeps": st.sweeps}
    if best is None:
        raise RuntimeError("no inner tolerance converged")
    if use_cache:
        _store(key, best)
    return dict(best, cached=False)
