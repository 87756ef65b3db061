import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def read_golden(name):
    """Parse a tests/golden fixture: returns dict with 'A', 'B', 'iters' {k: [x...]}, 'SOLUTION'."""
    out = {"iters": {}}
    with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, *vals = line.split()
            if head in ("A", "B", "SOLUTION"):
                out[head] = [float(v) for v in vals]
            else:
                out["iters"][int(head)] = [float(v) for v in vals]
    return out
