"""Host-side logic of the autotuner (no GPU): its result cache (atomic store, reload, a damaged file read as
empty) and that a cached workload is answered without timing anything."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1403_5805_gb300 import autotune  # noqa: E402


@pytest.fixture()
def cache(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("JACOBI_TUNE_CACHE", str(path))
    return path


def test_store_and_reload(cache):
    assert autotune._load_cache() == {}
    autotune._store("a", {"rows_per_warp": 4, "ms": 1.5})
    autotune._store("b", {"inner_rtol": 2.0 ** -10})
    assert json.loads(cache.read_text()) == {"a": {"rows_per_warp": 4, "ms": 1.5}, "b": {"inner_rtol": 2.0 ** -10}}
    autotune._store("a", {"rows_per_warp": 8, "ms": 1.0})  # a later result replaces the entry
    assert autotune._load_cache()["a"] == {"rows_per_warp": 8, "ms": 1.0}
    assert not [p for p in os.listdir(cache.parent) if ".tmp" in p]  # the temporary file was renamed


def test_damaged_cache_reads_as_empty(cache):
    cache.parent.mkdir(parents=True)
    cache.write_text("{not json")
    assert autotune._load_cache() == {}
    autotune._store("k", {"ms": 2.0})  # and is replaced by a valid file
    assert autotune._load_cache() == {"k": {"ms": 2.0}}


def test_cached_workload_is_not_timed(cache, monkeypatch):
    monkeypatch.setattr(autotune, "_signature", lambda kind, precision, sizes: f"{kind}|{precision}|{len(sizes)}")

    def no_timing(*a, **k):
        raise AssertionError("a cached workload must not be timed")

    monkeypatch.setattr(autotune, "_time", no_timing)
    autotune._store("batch|fp32_ir|3", {"rows_per_warp": 2, "ctas_per_sm": 4, "inner_rtol": 2.0 ** -10, "ms": 0.5})
    autotune._store("single|bf16_ir|1", {"inner_rtol": 2.0 ** -12, "ms": 2.4})

    class _A:
        def __init__(self, n):
            self.shape = (n, n)

    got = autotune.tune_batch([_A(10), _A(20), _A(30)], [None] * 3, precision="fp32_ir")
    assert got["cached"] and got["rows_per_warp"] == 2 and got["ctas_per_sm"] == 4
    got = autotune.tune_single(_A(100), None, "bf16_ir")
    assert got["cached"] and got["inner_rtol"] == 2.0 ** -12
