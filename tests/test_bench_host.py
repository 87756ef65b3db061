"""Host-side logic of bench.py (no GPU): the roofline arithmetic, the use of committed DRAM traffic, the
per-phase bandwidth of a device trace, and the job rate of N replicas (two gloo ranks on the CPU)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Props:
    multi_processor_count = 152


class _FakeTorch:
    class cuda:
        @staticmethod
        def get_device_properties(dev):
            return _Props()


PEAKS = {"hbm_gbs": 6793.1, "sm_max_mhz": 2070.0}


def test_composite_roofline_takes_the_larger_bound_per_phase():
    n = 16384
    main = {"kernel_ms": 2.4, "phases": {"resid64": {"count": 3, "mean_us": 494.5},
                                         "resid0": {"count": 1, "mean_us": 13.7},
                                         "inner": {"count": 5, "mean_us": 82.7},
                                         "narrow_inner": {"count": 1, "mean_us": 468.5}}}
    c = bench.composite_roofline(main, n, "bf16_ir", PEAKS, None, _FakeTorch)
    fma_s = 2.0 * 152 * 2070e6                     # FP64 FMAs per second
    t_resid = max(8.0 * n * n / 6793.1e9, n * n / fma_s)
    assert c["phases"]["resid64"]["bound"] == "fp64"  # FP64-FMA time exceeds the HBM time of 8 B per FMA
    assert c["phases"]["resid64"]["min_us"] == pytest.approx(t_resid * 1e6, abs=0.1)
    assert c["phases"]["inner"]["bound"] == "hbm"
    assert c["phases"]["inner"]["min_us"] == pytest.approx(2.0 * n * n / 6793.1e9 * 1e6, abs=0.1)
    assert c["phases"]["narrow_inner"]["min_us"] == pytest.approx(10.0 * n * n / 6793.1e9 * 1e6, abs=0.1)
    assert c["phases"]["resid0"]["min_us"] == 0.0
    total = 3 * t_resid + 5 * 2.0 * n * n / 6793.1e9 + 10.0 * n * n / 6793.1e9
    assert c["min_ms"] == pytest.approx(total * 1e3, abs=1e-3)
    assert c["frac"] == pytest.approx(total / 2.4e-3, abs=1e-3)


def test_composite_roofline_of_the_fp64_path():
    main = {"kernel_ms": 3.44, "phases": {"sweep64": {"count": 7, "mean_us": 488.6}}}
    c = bench.composite_roofline(main, 16384, "fp64", PEAKS, None, _FakeTorch)
    assert c["phases"]["sweep64"]["bound"] == "fp64" and c["phases"]["sweep64"]["count"] == 7
    assert 0.8 < c["frac"] < 0.95


def test_committed_traffic_needs_the_same_source_and_size(tmp_path, monkeypatch):
    record = {"k": {"source_sha256_16": "abc", "n": 16384, "dram_bytes_per_launch": 123}}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(record))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(path))
    monkeypatch.setattr(bench, "src_hash", lambda kernel="": "abc")
    assert bench.committed_traffic("k", 16384) == 123
    assert bench.committed_traffic("k", 8192) is None           # another size
    assert bench.committed_traffic("other", 16384) is None      # no record
    monkeypatch.setattr(bench, "src_hash", lambda kernel="": "changed")
    assert bench.committed_traffic("k", 16384) is None          # the kernel source changed since


def test_committed_traffic_file_is_current_for_its_kernels():
    """Every record in profiles/traffic.json names its size and source hash, and reads at most a few per
    mille above its algorithmic bytes (a capture far above them would mean re-reads)."""
    with open(bench.TRAFFIC_FILE) as fh:
        t = json.load(fh)
    for name, e in t.items():
        if name.startswith("_"):
            continue
        assert e["n"] == 16384 and len(e["source_sha256_16"]) == 16
        assert e["dram_bytes_per_launch"] == e["read"] + e["write"]
        assert 0.99 < e["dram_bytes_per_launch"] / e["algorithmic_bytes"] < 1.07, name


def test_phase_bandwidth_from_a_trace():
    n = 1000
    # kinds: resid0, fused first sweep, inner, inner, resid64 (ns)
    trace = [(2, 0, 1000), (4, 1000, 11000), (3, 11000, 13000), (3, 13000, 15000), (1, 15000, 35000)]
    ph = bench.phase_bandwidth(trace, n, "bf16_ir")
    assert ph["inner"]["count"] == 2 and ph["inner"]["mean_us"] == 2.0
    assert ph["inner"]["gbs"] == pytest.approx(2.0 * n * n / 2000.0, rel=1e-3)
    assert ph["narrow_inner"]["gbs"] == pytest.approx(10.0 * n * n / 10000.0, rel=1e-3)
    assert ph["resid64"]["gbs"] == pytest.approx(8.0 * n * n / 20000.0, rel=1e-3)
    assert ph["resid0"]["gbs"] is None


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms, rate = bench.job_rate(1.5 + rank, world, "cpu")  # rank 1 is the slower replica
        dist.barrier()
        out[rank] = (ms, rate)
    finally:
        dist.destroy_process_group()


def test_replica_job_rate_over_two_gloo_ranks():
    """bench.py --gpus N runs N replicas; the job's step time is the slowest rank's (MAX all-reduce) and
    the job's rate N / that time, on every rank.  Two CPU ranks over gloo."""
    torch = pytest.importorskip("torch")
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert dict(out) == {0: (2.5, 2 / 2.5e-3), 1: (2.5, 2 / 2.5e-3)}
    assert bench.job_rate(4.0, 1, "cpu") == (4.0, 250.0)
