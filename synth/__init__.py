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


def symmetric_system(n: int, f: float, seed: int, nrhs: int = 1):
    """Symmetric strictly diagonally dominant system with a planted solution: the off-diagonal entries of
    row i < j are the dominant generator's, mirrored below the diagonal (a_ji = a_ij), a_ii = f * sum_{j != i}
    |a_ij| * (+-1), so ||T||_inf = 1/f exactly.  Returns ``(A, B, Xstar)`` as dominant_system."""
    A = _offdiag(seed, n, signed=True)
    A = np.triu(A, 1)
    A = A + A.T                                    # exact: one of the two terms is zero
    rowsum = np.abs(A).sum(axis=1)                 # exact (integers times 2**-31)
    sign = np.where(random_u32(seed, STREAM_SIGN, n) & np.uint32(1), -1.0, 1.0)
    d = f * rowsum * sign
    if n == 1:
        d = np.array([f * sign[0]])
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


# ---- sparse (PDE-shaped) systems ------------------------------------------------------------------

def _csr_from_coo(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray):
    """CSR arrays (row_ptr int64, col_idx int32, values float64), columns ascending within each row."""
    order = np.argsort(rows.astype(np.int64) * n + cols, kind="stable")
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32), vals.astype(np.float64)


def _planted(seed: int, n: int, nrhs: int, row_ptr, col_idx, values):
    Xs = signed_unit(random_u32(seed, STREAM_XSTAR, n * nrhs)).reshape(nrhs, n).T.copy()
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    B = np.zeros((n, nrhs))
    for c in range(nrhs):  # B = A X* (input construction), summed row by row in column order
        B[:, c] = np.bincount(rows, weights=values * Xs[col_idx, c], minlength=n)
    return B, Xs


def stencil_system(shape, f: float, seed: int, nrhs: int = 1, weights: str = "variable", diag: str = "dominant"):
    """PDE-shaped sparse system: the 3-point (1-D), 5-point (2-D) or 7-point (3-D) stencil of a diffusion
    operator on a grid of ``shape`` with Dirichlet boundaries, unknowns numbered in row-major grid order
    (the Jacobi codes for differential equations that the paper's related work cites).

    Each grid edge e joining unknowns i and j carries a weight ``w_e`` and ``a_ij = a_ji = -w_e``.
    ``weights="variable"``: ``w_e = 1 + k_e 2**-20`` with ``k_e`` a uniform integer in [0, 2**20) (exact
    row sums); ``"unit"``: ``w_e = 1``.  ``diag="dominant"``: ``a_ii = f * sum_{j != i} w_ij``, so
    ``||T||_inf = 1/f`` exactly; ``"constant"``: ``a_ii = f * 2 * len(shape)`` on every row (the screened
    Poisson operator, whose Jacobi matrix has the grid's sine modes as eigenvectors).  Planted ``X*``
    uniform [-1, 1) and ``B = A X*``.

    Returns ``(row_ptr, col_idx, values, B, Xs)``: CSR with int64 row offsets, int32 columns strictly
    ascending within each row (the diagonal included) and FP64 values; B and X* ``(n, nrhs)``."""
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    grid = np.arange(n, dtype=np.int64).reshape(shape)
    lo_parts, hi_parts = [], []
    for ax in range(len(shape)):
        lo_parts.append(np.take(grid, np.arange(shape[ax] - 1), axis=ax).reshape(-1))
        hi_parts.append(np.take(grid, np.arange(1, shape[ax]), axis=ax).reshape(-1))
    lo = np.concatenate(lo_parts) if lo_parts else np.zeros(0, np.int64)
    hi = np.concatenate(hi_parts) if hi_parts else np.zeros(0, np.int64)
    if weights == "variable":
        w = 1.0 + (random_u32(seed, STREAM_A, lo.size) >> np.uint32(12)).astype(np.float64) * 2.0 ** -20
    else:
        w = np.ones(lo.size)
    if diag == "dominant":
        rowsum = np.bincount(lo, weights=w, minlength=n) + np.bincount(hi, weights=w, minlength=n)
        d = f * rowsum
        d[rowsum == 0] = f  # an isolated unknown (a grid of one point)
    else:
        d = np.full(n, f * 2.0 * len(shape))
    diag_idx = np.arange(n, dtype=np.int64)
    row_ptr, col_idx, values = _csr_from_coo(n, np.concatenate([lo, hi, diag_idx]), np.concatenate([hi, lo, diag_idx]),
                                             np.concatenate([-w, -w, d]))
    B, Xs = _planted(seed, n, nrhs, row_ptr, col_idx, values)
    return row_ptr, col_idx, values, B, Xs


def random_sparse_system(n: int, f: float, seed: int, max_len: int = 64, nrhs: int = 1):
    """Irregular sparse system: row i draws ``L_i`` off-diagonal positions (``L_i`` log-uniform in
    [1, max_len + 1] minus one, so most rows are short, some empty and a few long) at uniform random
    columns other than i (repeats merged), values ``int32(w) 2**-31`` in [-1, 1), and
    ``a_ii = f * sum_{j != i} |a_ij| * (+-1)`` (``+-f`` for a row without off-diagonals).
    Returns ``(row_ptr, col_idx, values, B, Xs)`` as ``stencil_system``."""
    u = unit(random_u32(seed, STREAM_META, n))
    L = log_uniform_int(u, 1, max_len + 1) - 1 if n > 1 else np.zeros(n, np.int64)
    rows = np.repeat(np.arange(n, dtype=np.int64), L)
    m = rows.size
    pos = random_u32(seed, STREAM_A, 2 * m).reshape(m, 2) if m else np.zeros((0, 2), np.uint32)
    cols = pos[:, 0].astype(np.int64) % max(n - 1, 1)
    cols = cols + (cols >= rows)  # skip the diagonal
    key, first = np.unique(rows * n + cols, return_index=True)
    rows, cols = key // n, key % n
    vals = signed_unit(pos[first, 1])
    vals[vals == 0.0] = 2.0 ** -31  # keep every stored off-diagonal non-zero
    rowsum = np.bincount(rows, weights=np.abs(vals), minlength=n)
    sign = np.where(random_u32(seed, STREAM_SIGN, n) & np.uint32(1), -1.0, 1.0)
    d = np.where(rowsum > 0, f * rowsum, f) * sign
    diag_idx = np.arange(n, dtype=np.int64)
    row_ptr, col_idx, values = _csr_from_coo(n, np.concatenate([rows, diag_idx]), np.concatenate([cols, diag_idx]),
                                             np.concatenate([vals, d]))
    B, Xs = _planted(seed, n, nrhs, row_ptr, col_idx, values)
    return row_ptr, col_idx, values, B, Xs


def csr_to_dense(n: int, row_ptr, col_idx, values) -> np.ndarray:
    """The dense row-major matrix of a CSR one (for the tests)."""
    A = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    A[rows, col_idx] = values
    return A
