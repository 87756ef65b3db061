"""Plain FP64 CPU oracle of the dense Jacobi solver (arXiv:1403.5805, Section 2).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path: the arithmetic lives in
``jacobi_oracle.c`` (plain C loops, FP64), compiled here with gcc; this module only marshals numpy arrays.

Layouts: A is row-major ``(n, n)``; B and X are ``(n, nrhs)`` numpy arrays whose columns are the
right-hand sides (stored column-major for the C code, i.e. ``X[:, c]`` contiguous in the C buffer).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jacobi_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, NOT_CONVERGED, INVALID_ARG, ZERO_DIAGONAL, NONFINITE, NO_MEMORY = 0, 1, -1, -2, -3, -4
NORM_INF, NORM_2, NORM_RESID = 0, 1, 2

_c_i64 = ctypes.c_int64
_c_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile ``jacobi_oracle.c`` into ``_build/liboracle.so`` (gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp = ctypes.c_void_p
            lib.oracle_jacobi.argtypes = [_c_i64, _c_i64, vp, vp, vp, _c_i64, ctypes.c_double,
                                          ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(_c_i64),
                                          _c_dp, vp]
            lib.oracle_jacobi.restype = ctypes.c_int
            lib.oracle_block_sor.argtypes = [_c_i64, _c_i64, vp, vp, vp, _c_i64, ctypes.c_double, ctypes.c_int,
                                             _c_i64, vp, ctypes.c_double, vp, ctypes.POINTER(_c_i64), _c_dp, vp]
            lib.oracle_block_sor.restype = ctypes.c_int
            lib.oracle_csr_jacobi.argtypes = [_c_i64, vp, vp, vp, vp, vp, _c_i64, ctypes.c_double, ctypes.c_int,
                                              vp, ctypes.POINTER(_c_i64), _c_dp, vp]
            lib.oracle_csr_jacobi.restype = ctypes.c_int
            lib.oracle_csr_residual.argtypes = [_c_i64, vp, vp, vp, vp, vp, vp, _c_dp]
            lib.oracle_csr_residual.restype = ctypes.c_int
            lib.oracle_ge.argtypes = [_c_i64, _c_i64, vp, vp, vp]
            lib.oracle_ge.restype = ctypes.c_int
            lib.oracle_residual.argtypes = [_c_i64, _c_i64, vp, vp, vp, vp, _c_dp]
            lib.oracle_residual.restype = ctypes.c_int
            lib.oracle_residual_rows.argtypes = [_c_i64, _c_i64, vp, vp, vp, _c_i64, vp, vp]
            lib.oracle_residual_rows.restype = ctypes.c_int
            lib.oracle_split.argtypes = [_c_i64, _c_i64, vp, vp, vp, vp]
            lib.oracle_split.restype = ctypes.c_int
            lib.oracle_bf16_from_f32.argtypes = [ctypes.c_float]
            lib.oracle_bf16_from_f32.restype = ctypes.c_uint16
            lib.oracle_e4m3_from_f32.argtypes = [ctypes.c_float]
            lib.oracle_e4m3_from_f32.restype = ctypes.c_uint8
            lib.oracle_offdiag_f32.argtypes = [_c_i64, vp, vp]
            lib.oracle_offdiag_bf16.argtypes = [_c_i64, vp, vp]
            lib.oracle_offdiag_e4m3.argtypes = [_c_i64, vp, vp, vp]
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _mat(A) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be square")
    return A


def _cols(B, n) -> np.ndarray:
    """(n,) or (n, r) array -> column-major buffer as an (r, n) C-contiguous array."""
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    if B.shape[0] != n:
        raise ValueError("row count mismatch")
    return np.ascontiguousarray(B.T)


@dataclass
class JacobiResult:
    status: int
    X: np.ndarray          # (n, nrhs)
    iters: int
    delta: float
    trace: np.ndarray | None  # (iters, n, nrhs) iterates X^(1..iters), if requested


def jacobi(A, B, X0=None, max_iter: int = 1000, tol: float = 1e-12, norm: int = NORM_INF,
           nthreads: int = 1, trace: bool = False) -> JacobiResult:
    """Section 2 Jacobi iteration on the CPU in FP64 (component form, ascending-j sums)."""
    lib = _load()
    A = _mat(A)
    n = A.shape[0]
    Bc = _cols(B, n)
    r = Bc.shape[0]
    X0c = None if X0 is None else _cols(X0, n)
    Xo = np.zeros((r, n))
    it = _c_i64(0)
    de = ctypes.c_double(0.0)
    tr = np.zeros((max_iter, r, n)) if trace else None
    st = lib.oracle_jacobi(n, r, _ptr(A), _ptr(Bc), None if X0c is None else _ptr(X0c), max_iter,
                           tol, norm, nthreads, _ptr(Xo), ctypes.byref(it), ctypes.byref(de),
                           None if tr is None else _ptr(tr))
    k = int(it.value)
    tr_out = None if tr is None else np.ascontiguousarray(tr[:k].transpose(0, 2, 1))
    return JacobiResult(st, Xo.T.copy(), k, float(de.value), tr_out)


def uniform_blocks(n: int, nblocks: int) -> np.ndarray:
    """Offsets of nblocks consecutive row blocks of near-equal size: s_b = floor(n b / nblocks)."""
    return np.array([n * b // nblocks for b in range(nblocks + 1)], dtype=np.int64)


def block_sor(A, B, X0=None, max_iter: int = 1000, tol: float = 1e-12, norm: int = NORM_INF,
              blocks=1, omega: float = 1.0, trace: bool = False) -> JacobiResult:
    """Block-hybrid Gauss-Seidel / SOR (Gauss-Seidel inside consecutive row blocks, Jacobi across them,
    relaxation omega) on the CPU in FP64.  blocks: a block count (uniform split) or the offsets."""
    lib = _load()
    A = _mat(A)
    n = A.shape[0]
    Bc = _cols(B, n)
    r = Bc.shape[0]
    starts = uniform_blocks(n, int(blocks)) if np.isscalar(blocks) else np.ascontiguousarray(blocks, dtype=np.int64)
    X0c = None if X0 is None else _cols(X0, n)
    Xo = np.zeros((r, n))
    it = _c_i64(0)
    de = ctypes.c_double(0.0)
    tr = np.zeros((max_iter, r, n)) if trace else None
    st = lib.oracle_block_sor(n, r, _ptr(A), _ptr(Bc), None if X0c is None else _ptr(X0c), max_iter, tol, norm,
                              len(starts) - 1, starts.ctypes.data_as(ctypes.c_void_p), ctypes.c_double(omega),
                              _ptr(Xo), ctypes.byref(it), ctypes.byref(de), None if tr is None else _ptr(tr))
    k = int(it.value)
    tr_out = None if tr is None else np.ascontiguousarray(tr[:k].transpose(0, 2, 1))
    return JacobiResult(st, Xo.T.copy(), k, float(de.value), tr_out)


def csr_jacobi(row_ptr, col_idx, values, B, X0=None, max_iter: int = 1000, tol: float = 1e-12,
               norm: int = NORM_INF, trace: bool = False) -> JacobiResult:
    """Section 2 Jacobi iteration for a sparse A in CSR (int64 row offsets, int32 columns strictly
    ascending within each row, the diagonal among them), one right-hand side, on the CPU in FP64."""
    lib = _load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    va = np.ascontiguousarray(values, dtype=np.float64)
    n = rp.size - 1
    b = np.ascontiguousarray(np.asarray(B, dtype=np.float64).reshape(-1))
    if b.size != n or ci.size != va.size or n < 1 or rp[-1] != ci.size:
        raise ValueError("CSR shape mismatch")
    x0 = None if X0 is None else np.ascontiguousarray(np.asarray(X0, dtype=np.float64).reshape(-1))
    Xo = np.zeros(n)
    it = _c_i64(0)
    de = ctypes.c_double(0.0)
    tr = np.zeros((max_iter, n)) if trace else None
    st = lib.oracle_csr_jacobi(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(b), None if x0 is None else _ptr(x0), max_iter,
                               tol, norm, _ptr(Xo), ctypes.byref(it), ctypes.byref(de), None if tr is None else _ptr(tr))
    k = int(it.value)
    return JacobiResult(st, Xo[:, None].copy(), k, float(de.value), None if tr is None else tr[:k, :, None].copy())


def csr_residual(row_ptr, col_idx, values, B, X) -> tuple[np.ndarray, float]:
    """r = b - A x for a CSR matrix (FP64, stored entries in column order) and ||r||_inf / ||b||_inf."""
    lib = _load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    va = np.ascontiguousarray(values, dtype=np.float64)
    n = rp.size - 1
    b = np.ascontiguousarray(np.asarray(B, dtype=np.float64).reshape(-1))
    x = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(-1))
    if b.size != n or x.size != n:
        raise ValueError("vector length mismatch")
    R = np.zeros(n)
    rel = ctypes.c_double(0.0)
    lib.oracle_csr_residual(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(b), _ptr(x), _ptr(R), ctypes.byref(rel))
    return R, float(rel.value)


def ge(A, B) -> tuple[int, np.ndarray]:
    """Gaussian elimination with partial pivoting.  Returns (status, X)."""
    lib = _load()
    A = _mat(A)
    n = A.shape[0]
    Bc = _cols(B, n)
    X = np.zeros_like(Bc)
    st = lib.oracle_ge(n, Bc.shape[0], _ptr(A), _ptr(Bc), _ptr(X))
    return st, X.T.copy()


def residual(A, B, X) -> tuple[np.ndarray, float]:
    """R = B - A X (FP64) and the relative residual max_c ||r_c||_inf / ||b_c||_inf."""
    lib = _load()
    A = _mat(A)
    n = A.shape[0]
    Bc = _cols(B, n)
    Xc = _cols(X, n)
    R = np.zeros_like(Bc)
    rel = ctypes.c_double(0.0)
    lib.oracle_residual(n, Bc.shape[0], _ptr(A), _ptr(Bc), _ptr(Xc), _ptr(R), ctypes.byref(rel))
    return R.T.copy(), float(rel.value)


def residual_rows(A, B, X, rows) -> np.ndarray:
    """R[t, c] = B[i, c] - sum_j A[i, j] X[j, c] for i = rows[t] (FP64, the same row sums as residual())."""
    lib = _load()
    A = _mat(A)
    n = A.shape[0]
    Bc = _cols(B, n)
    Xc = _cols(X, n)
    rw = np.ascontiguousarray(rows, dtype=np.int64)
    R = np.zeros((Bc.shape[0], rw.size))
    st = lib.oracle_residual_rows(n, Bc.shape[0], _ptr(A), _ptr(Bc), _ptr(Xc), rw.size, _ptr(rw), _ptr(R))
    if st != OK:
        raise ValueError("invalid rows")
    return R.T.copy()


def split(A, B) -> tuple[int, np.ndarray, np.ndarray]:
    """Fixed-point form T = D^-1 (L + U), C = D^-1 B.  Returns (status, T, C)."""
    lib = _load()
    A = _mat(A)
    n = A.shape[0]
    Bc = _cols(B, n)
    T = np.zeros_like(A)
    C = np.zeros_like(Bc)
    st = lib.oracle_split(n, Bc.shape[0], _ptr(A), _ptr(Bc), _ptr(T), _ptr(C))
    return st, T, C.T.copy()


def bf16_from_f32(x: float) -> int:
    return int(_load().oracle_bf16_from_f32(float(x)))


def e4m3_from_f32(x: float) -> int:
    return int(_load().oracle_e4m3_from_f32(float(x)))


def offdiag_f32(A) -> np.ndarray:
    A = _mat(A)
    out = np.zeros(A.shape, dtype=np.float32)
    _load().oracle_offdiag_f32(A.shape[0], _ptr(A), _ptr(out))
    return out


def offdiag_bf16(A) -> np.ndarray:
    """BF16 codes (uint16) of the off-diagonal part of A."""
    A = _mat(A)
    out = np.zeros(A.shape, dtype=np.uint16)
    _load().oracle_offdiag_bf16(A.shape[0], _ptr(A), _ptr(out))
    return out


def offdiag_e4m3(A) -> tuple[np.ndarray, np.ndarray]:
    """E4M3 codes (uint8) and FP32 row scales of the off-diagonal part of A."""
    A = _mat(A)
    n = A.shape[0]
    q = np.zeros(A.shape, dtype=np.uint8)
    s = np.zeros(n, dtype=np.float32)
    _load().oracle_offdiag_e4m3(n, _ptr(A), _ptr(q), _ptr(s))
    return q, s


def num_threads() -> int:
    return int(_load().oracle_num_threads())
