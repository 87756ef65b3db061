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


def f64_narrowing_cases(seed=0, random_count=4000):
    """FP64 values whose FP64 -> FP32 rounding takes every branch: exact values, ties to even at the 29
    dropped fraction bits, carries into the exponent and to infinity, FP32 subnormals (ties included),
    underflow to signed zero, FP64 subnormals and infinities; then random bit patterns whose exponents
    span FP32's subnormal, normal and overflow ranges (no NaN)."""
    import numpy as np
    flt_max = (2.0 - 2.0 ** -23) * 2.0 ** 127
    fixed = [0.0, -0.0, 1.0, -1.0, 0.1, -3.7,
             1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24, 1 + 2.0 ** -24 + 2.0 ** -52, 1 - 2.0 ** -25,
             1 - 2.0 ** -25 - 2.0 ** -53, 2 - 2.0 ** -24, -(2 - 2.0 ** -24),
             flt_max, -flt_max, flt_max + 2.0 ** 103, flt_max + 2.0 ** 103 - 2.0 ** 75, 2.0 ** 128, 1e300, -1e300,
             float("inf"), float("-inf"),
             2.0 ** -126, 2.0 ** -126 - 2.0 ** -150, 2.0 ** -126 - 2.0 ** -150 - 2.0 ** -160,
             2.0 ** -149, 2.0 ** -150, 2.0 ** -150 + 2.0 ** -170, 3 * 2.0 ** -150, 5 * 2.0 ** -150,
             -3 * 2.0 ** -150, 2.0 ** -151, 1.5 * 2.0 ** -140, 1e-300, -1e-300, 5e-324, -5e-324, 2.0 ** -1022]
    rng = np.random.default_rng(seed)
    frac = rng.integers(0, 1 << 52, random_count, dtype=np.uint64)
    frac[: random_count // 4] &= ~np.uint64((1 << 29) - 1)            # exact in FP32 ...
    frac[: random_count // 8] |= np.uint64(1 << 28)                    # ... or exactly half-way
    exp = rng.integers(896 - 40, 896 + 260, random_count).astype(np.uint64)
    sign = rng.integers(0, 2, random_count).astype(np.uint64) << np.uint64(63)
    rand = (sign | (exp << np.uint64(52)) | frac).view(np.float64)
    return np.concatenate([np.array(fixed, dtype=np.float64), rand])
