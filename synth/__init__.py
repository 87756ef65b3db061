"""Seeded synthetic inputs for the dense Jacobi solver (shared by the oracle tests, the CUDA-path tests
and the benchmark).

This module holds no arithmetic of the Jacobi method itself: it only draws matrices and vectors.  Every
random number comes from Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11), a counter-based generator, so that any element can be regenerated from
``(seed, stream, index)`` alone, on the host here or by a device-side twin of the same published
definition.

Workload shapes (the paper's Section 4 uses dense random A, B, X in [0, 1]; the solver configs add
strictly diagonally dominant variants, Section 2's convergence condition):

* ``dominant_system``  off-diagonals iid uniform [-1, 1), ``a_ii = f * sum_{j!=i} |a_ij| * (+-1)``, so
  ``||T||_inf = 1/f`` exactly; planted ``X*`` iid uniform [-1, 1) and ``B = A X*``.
* ``hard_system``      the paper-shaped generator: off-diagonals uniform [0, 1), positive diagonal
  ``a_ii = f * sum_{j!=i} a_ij``.  Then ``T = -(1/f) S`` with ``S`` row-stochastic, so the spectral
  radius of T is exactly ``1/f`` and Jacobi needs ``~ ln(tol)/ln(1/f)`` sweeps.

Off-diagonal entries are integers times ``2**-31`` (or ``2**-32``), so every row sum of ``|a_ij|`` with
``n <= 2**21`` is exact in FP64 whatever the summation order.
"""
from __future__ import annotations

import math

import numpy as np

# Philox4x32-10 constants (Salmon et al., SC'11, Section 5 / Table 2): multipliers and Weyl key bumps.
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint32(0x9E3779B9)
_PHILOX_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)

BASE_SEED = 14035805


def philox4x32_10(ctr: np.ndarray, key: tuple[int, int]) -> np.ndarray:
    """Philox4x32 with 10 rounds.  ``ctr`` is a ``(N, 4)`` uint32 array of counters, ``key`` two uint32
    words.  Returns ``(N, 4)`` uint32 outputs."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).astype(np.uint64)
    c0, c1, c2, c3 = c[:, 0].copy(), c[:, 1].copy(), c[:, 2].copy(), c[:, 3].copy()
    k0 = np.uint32(key[0] & 0xFFFFFFFF)
    k1 = np.uint32(key[1] & 0xFFFFFFFF)
    for r in range(10):
        p0 = _PHILOX_M0 * c0          # 64-bit product of two 32-bit words (no overflow in uint64)
        p1 = _PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0)), lo1, (hi0 ^ c3 ^ np.uint64(k1)), lo0
        if r != 9:
            k0 = np.uint32((int(k0) + int(_PHILOX_W0)) & 0xFFFFFFFF)
            k1 = np.uint32((int(k1) + int(_PHILOX_W1)) & 0xFFFFFFFF)
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def _blocks(seed: int, stream: int, first: int, last: int) -> np.ndarray:
    q = np.arange(first, last + 1, dtype=np.uint64)
    ctr = np.zeros((q.size, 4), dtype=np.uint32)
    ctr[:, 0] = (q & _MASK32).astype(np.uint32)
    ctr[:, 1] = (q >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = np.uint32(stream & 0xFFFFFFFF)
    return philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)).reshape(-1)


_PAR_BLOCKS = 1 << 20  # split larger requests over threads (numpy releases the GIL in its kernels)


def random_u32(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` uint32 words of the sequence ``(seed, stream)`` starting at word ``offset``.

    Word ``w`` is output lane ``w % 4`` of the Philox block with counter
    ``(w // 4 mod 2**32, w // 4 >> 32, stream, 0)`` and key ``(seed mod 2**32, seed >> 32)``."""
    if count <= 0:
        return np.zeros(0, dtype=np.uint32)
    first = offset // 4
    last = (offset + count - 1) // 4
    nblk = last - first + 1
    if nblk <= _PAR_BLOCKS:
        out = _blocks(seed, stream, first, last)
    else:
        import concurrent.futures as cf
        import os
        out = np.empty(nblk * 4, dtype=np.uint32)
        step = _PAR_BLOCKS

        def work(a):
            b = min(a + step, nblk) - 1
            out[4 * a:4 * (b + 1)] = _blocks(seed, stream, first + a, first + b)

        with cf.ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 1)) as ex:
            list(ex.map(work, range(0, nblk, step)))
    start = offset - first * 4
    return out[start:start + count]


def signed_unit(words: np.ndarray) -> np.ndarray:
    """uint32 words -> FP64 values ``int32(w) * 2**-31`` in [-1, 1) (exact)."""
    return words.view(np.int32).astype(np.float64) * (2.0 ** -31)


def unit(words: np.ndarray) -> np.ndarray:
    """uint32 words -> FP64 values ``w * 2**-32`` in [0, 1) (exact)."""
    return words.astype(np.float64) * (2.0 ** -32)


# Stream ids inside one system's seed.
STREAM_A, STREAM_SIGN, STREAM_XSTAR, STREAM_X0, STREAM_META, STREAM_B = 0, 1, 2, 3, 4, 5


def _offdiag(seed: int, n: int, signed: bool) -> np.ndarray:
    w = random_u32(seed, STREAM_A, n * n).reshape(n, n)
    A = signed_unit(w) if signed else unit(w)
    np.fill_diagonal(A, 0.0)
    return A


def dominant_system(n: int, f: float, seed: int, nrhs: int = 1):
    """Strictly diagonally dominant system with a planted solution.

    Returns ``(A, B, Xstar)``: A row-major ``(n, n)`` FP64, B and X* ``(n, nrhs)`` FP64 (column ``c`` is
    right-hand side ``c``)."""
    A = _offdiag(seed, n, signed=True)
    rowsum = np.abs(A).sum(axis=1)                 # exact (integers times 2**-31)
    sign = np.where(random_u32(seed, STREAM_SIGN, n) & np.uint32(1), -1.0, 1.0)
    d = f * rowsum * sign
    if n == 1:
        d = np.array([f * sign[0]])                 # a 1x1 system has no off-diagonals
    A[np.arange(n), np.arange(n)] = d
    Xs = signed_unit(random_u32(seed, STREAM_XSTAR, n * nrhs)).reshape(nrhs, n).T.copy()
    B = A @ Xs
    return A, B, Xs


def hard_system(n: int, f: float, seed: int, nrhs: int = 1):
    """The paper-shaped generator (Section 4 draws entries uniformly from [0, 1]) made convergent: a
    positive diagonal ``f`` times the row sum.  ``rho(T) = ||T||_inf = 1/f``.  Returns ``(A, B, Xstar)``."""
    A = _offdiag(seed, n, signed=False)
    d = f * A.sum(axis=1)
    if n == 1:
        d = np.array([f])
    A[np.arange(n), np.arange(n)] = d
    Xs = signed_unit(random_u32(seed, STREAM_XSTAR, n * nrhs)).reshape(nrhs, n).T.copy()
    B = A @ Xs
    return A, B, Xs


def log_uniform_int(u: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Map uniforms in [0, 1) to integers log-uniform on [lo, hi]."""
    v = np.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo)))
    return np.clip(np.floor(v).astype(np.int64), lo, hi)


def batch_shapes(count: int, n_lo: int, n_hi: int, f_lo: float, f_hi: float, seed: int):
    """Sizes ``n`` (log-uniform on [n_lo, n_hi]) and dominance factors ``f`` (uniform on [f_lo, f_hi])
    of ``count`` independent systems."""
    u = unit(random_u32(seed, STREAM_META, 2 * count)).reshape(count, 2)
    n = log_uniform_int(u[:, 0], n_lo, n_hi)
    f = f_lo + u[:, 1] * (f_hi - f_lo)
    return n, f


def system_seed(seed: int, index: int) -> int:
    """Seed of system ``index`` in a batch drawn with ``seed``."""
    return (seed * 1_000_003 + index + 1) & 0xFFFFFFFFFFFF


def serving_request(n: int, nrhs: int, f: float, seed: int):
    """One request of the serving workload: the dominant generator's A (off-diagonals int32(w) * 2**-31,
    a_ii = f * sum_{j != i} |a_ij| * (+-1)) and right-hand sides drawn directly, B iid uniform [-1, 1)
    (word c * n + i of stream 5 is B[i, c]).  Every value is a function of (seed, stream, index) alone,
    so a device-side twin of the same generator reproduces A and B bit for bit.  Returns (A, B)."""
    A = _offdiag(seed, n, signed=True)
    rowsum = np.abs(A).sum(axis=1)  # exact: integers times 2**-31, the zero diagonal included
    sign = np.where(random_u32(seed, STREAM_SIGN, n) & np.uint32(1), -1.0, 1.0)
    A[np.arange(n), np.arange(n)] = f * rowsum * sign if n > 1 else np.array([f * sign[0]])
    B = signed_unit(random_u32(seed, STREAM_B, n * nrhs)).reshape(nrhs, n).T.copy()
    return A, B


def serving_trace(rate: float, duration: float, seed: int, n_lo: int = 256, n_hi: int = 8192, r_max: int = 16,
                  f_lo: float = 1.05, f_hi: float = 1.5):
    """Poisson arrivals at `rate` per second for `duration` seconds: arrays (t, n, r, f, seed) of the
    requests (exponential gaps from uniforms, n log-uniform in [n_lo, n_hi], r uniform in {1..r_max},
    f uniform in [f_lo, f_hi])."""
    count = int(rate * duration * 1.5) + 16
    u = unit(random_u32(seed, STREAM_META, 4 * count)).reshape(count, 4)
    gaps = -np.log1p(-u[:, 0]) / rate
    t = np.cumsum(gaps)
    keep = t < duration
    t, u = t[keep], u[keep]
    n = log_uniform_int(u[:, 1], n_lo, n_hi)
    r = np.minimum((u[:, 2] * r_max).astype(np.int64) + 1, r_max)
    f = f_lo + u[:, 3] * (f_hi - f_lo)
    seeds = np.array([system_seed(seed, k) for k in range(len(t))], dtype=np.int64)
    return t, n, r, f, seeds
