"""ctypes binding of ``libjacobi.so`` (the C ABI in ``include/jacobi.h``).

Argument marshalling only: every step of a solve runs in the library's CUDA kernels.  There is no CPU
fallback; if the library has not been built, loading it raises.  PyTorch is used for device memory and
streams (the workspace tensor, the caller's stream), nothing else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libjacobi.so")

# jacobi_status
OK, NOT_CONVERGED = 0, 1
ERR_INVALID_ARG, ERR_ZERO_DIAGONAL, ERR_NONFINITE, ERR_OUT_OF_MEMORY = -1, -2, -3, -4
ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = -5, -6, -8
# jacobi_precision
FP64, FP32_IR, BF16_IR, FP8_IR = 0, 1, 2, 3
PRECISIONS = {"fp64": FP64, "fp32_ir": FP32_IR, "bf16_ir": BF16_IR, "fp8_ir": FP8_IR}
# jacobi_norm
NORM_INF, NORM_2, NORM_RESID = 0, 1, 2
# trace phase kinds (JACOBI_PHASE_*)
PHASE_SWEEP64, PHASE_RESID64, PHASE_RESID0, PHASE_INNER, PHASE_NARROW_INNER = 0, 1, 2, 3, 4
NORMS = {"inf": NORM_INF, "2": NORM_2, "resid": NORM_RESID}
FLAG_COPY_A = 1
FLAG_SPLIT_RESIDUAL = 2
FLAG_SHORT_WAITS = 4
FLAG_TEST_DROP_COPY = 8
FLAG_TEST_SKIP_ARRIVAL = 32
FLAG_CSR_ELL = 64  # sparse handle: keep sliced ELL even for a banded matrix
FLAG_RETIRE_COLUMNS = 16
FLAG_TC_RESIDUAL = 128
FLAG_SYMMETRIC = 256
METHODS = {"jacobi": 0, "sor": 1}

EXPORTS = ("jacobi_setup", "jacobi_solve", "jacobi_destroy", "jacobi_status_string", "jacobi_last_cuda_error",
           "jacobi_desc_init", "jacobi_workspace_size", "jacobi_setup_ex", "jacobi_solve_async",
           "jacobi_solve_ex", "jacobi_last_stats", "jacobi_residual", "jacobi_get_narrow",
           "jacobi_last_trace", "jacobi_column_stats", "jacobi_solve_fp64_noalloc", "jacobi_batch_workspace_size",
           "jacobi_batch_create", "jacobi_batch_solve_async", "jacobi_batch_stats", "jacobi_batch_grid",
           "jacobi_batch_destroy", "jacobi_server_create", "jacobi_server_submit", "jacobi_server_submit_generated",
           "jacobi_server_step", "jacobi_server_poll", "jacobi_server_rounds", "jacobi_server_destroy",
           "jacobi_generate_request", "jacobi_csr_setup", "jacobi_csr_solve_async", "jacobi_csr_solve",
           "jacobi_csr_last_stats", "jacobi_csr_info", "jacobi_csr_last_trace", "jacobi_csr_destroy",
           "jacobi_batch_solve", "jacobi_server_wait", "jacobi_csr_format", "jacobi_measure_fma_rates")


class JacobiStats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("outer_steps", ctypes.c_int64), ("final_delta", ctypes.c_double),
                ("rel_residual", ctypes.c_double), ("status", ctypes.c_int32), ("converged", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class JacobiBatchDesc(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64), ("n", ctypes.c_void_p), ("A", ctypes.c_void_p), ("B", ctypes.c_void_p),
                ("X", ctypes.c_void_p), ("precision", ctypes.c_int32), ("rows_per_warp", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("max_outer", ctypes.c_int32), ("max_inner", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("inner_rtol", ctypes.c_double), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("stream", ctypes.c_void_p)]


class JacobiServerDesc(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int64),
                ("max_inner", ctypes.c_int32), ("max_outer", ctypes.c_int32), ("inner_rtol", ctypes.c_double),
                ("max_active", ctypes.c_int32), ("flags", ctypes.c_int32), ("stream", ctypes.c_void_p)]


class JacobiDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nrhs", ctypes.c_int64), ("precision", ctypes.c_int32),
                ("norm", ctypes.c_int32), ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("stream", ctypes.c_void_p), ("grid", ctypes.c_int32),
                ("max_outer", ctypes.c_int32), ("inner_rtol", ctypes.c_double), ("max_inner", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("method", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("omega", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


class JacobiCsrDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("values", ctypes.c_void_p), ("B", ctypes.c_void_p),
                ("norm", ctypes.c_int32), ("flags", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("precision", ctypes.c_int32), ("max_outer", ctypes.c_int32), ("max_inner", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("inner_rtol", ctypes.c_double)]


class JacobiError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.jacobi_status_string(status).decode()
        cuda = lib.jacobi_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} ({status})" + (f" [{cuda}]" if cuda else ""))
        self.status = status


def load() -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built ({LIB_PATH}); run __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        H = ctypes.c_void_p
        lib.jacobi_setup.argtypes = [vp, vp, i64, ctypes.POINTER(H)]
        lib.jacobi_solve.argtypes = [H, vp, i64, dbl, vp, ctypes.POINTER(i64), ctypes.POINTER(dbl)]
        lib.jacobi_destroy.argtypes = [H]
        lib.jacobi_destroy.restype = None
        lib.jacobi_status_string.argtypes = [i32]
        lib.jacobi_status_string.restype = ctypes.c_char_p
        lib.jacobi_last_cuda_error.restype = ctypes.c_char_p
        lib.jacobi_desc_init.argtypes = [ctypes.POINTER(JacobiDesc)]
        lib.jacobi_desc_init.restype = None
        lib.jacobi_workspace_size.argtypes = [ctypes.POINTER(JacobiDesc), ctypes.POINTER(ctypes.c_size_t)]
        lib.jacobi_setup_ex.argtypes = [ctypes.POINTER(JacobiDesc), ctypes.POINTER(H)]
        lib.jacobi_solve_async.argtypes = [H, vp, i64, dbl, vp, vp]
        lib.jacobi_solve_ex.argtypes = [H, vp, i64, dbl, vp, ctypes.POINTER(JacobiStats)]
        lib.jacobi_last_stats.argtypes = [H, ctypes.POINTER(JacobiStats)]
        lib.jacobi_residual.argtypes = [H, vp, ctypes.POINTER(dbl)]
        lib.jacobi_get_narrow.argtypes = [H, vp, i64, vp]
        lib.jacobi_last_trace.argtypes = [H, vp, vp, i32, ctypes.POINTER(ctypes.c_int32)]
        lib.jacobi_column_stats.argtypes = [H, vp, vp]
        lib.jacobi_batch_workspace_size.argtypes = [ctypes.POINTER(JacobiBatchDesc), ctypes.POINTER(ctypes.c_size_t)]
        lib.jacobi_batch_create.argtypes = [ctypes.POINTER(JacobiBatchDesc), ctypes.POINTER(H)]
        lib.jacobi_batch_solve_async.argtypes = [H, i64, dbl]
        lib.jacobi_batch_stats.argtypes = [H, vp]
        lib.jacobi_batch_grid.argtypes = [H]
        lib.jacobi_batch_destroy.argtypes = [H]
        lib.jacobi_batch_destroy.restype = None
        lib.jacobi_server_create.argtypes = [ctypes.POINTER(JacobiServerDesc), ctypes.POINTER(H)]
        lib.jacobi_server_submit.argtypes = [H, i64, i64, vp, vp, vp, ctypes.POINTER(i64)]
        lib.jacobi_server_submit_generated.argtypes = [H, i64, i64, dbl, ctypes.c_uint64, vp, ctypes.POINTER(i64)]
        lib.jacobi_server_step.argtypes = [H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
        lib.jacobi_server_poll.argtypes = [H, vp, vp, i32, ctypes.POINTER(ctypes.c_int32)]
        lib.jacobi_server_rounds.argtypes = [H, ctypes.POINTER(i64)]
        lib.jacobi_server_destroy.argtypes = [H]
        lib.jacobi_server_destroy.restype = None
        lib.jacobi_generate_request.argtypes = [i64, i64, dbl, ctypes.c_uint64, vp, vp, i64, vp]
        lib.jacobi_solve_fp64_noalloc.argtypes = [vp, i64, vp, i64, vp, i64, dbl, vp, ctypes.POINTER(JacobiStats), vp]
        lib.jacobi_csr_setup.argtypes = [ctypes.POINTER(JacobiCsrDesc), ctypes.POINTER(H)]
        lib.jacobi_csr_solve_async.argtypes = [H, vp, i64, dbl, vp]
        lib.jacobi_csr_solve.argtypes = [H, vp, i64, dbl, vp, ctypes.POINTER(JacobiStats)]
        lib.jacobi_csr_last_stats.argtypes = [H, ctypes.POINTER(JacobiStats)]
        lib.jacobi_csr_info.argtypes = [H, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32)]
        lib.jacobi_csr_format.argtypes = [H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
        lib.jacobi_csr_last_trace.argtypes = [H, vp, vp, i32, ctypes.POINTER(ctypes.c_int32)]
        lib.jacobi_batch_solve.argtypes = [i64, vp, vp, vp, vp, dbl, i64, i32, vp]
        lib.jacobi_server_wait.argtypes = [H, i64, ctypes.POINTER(JacobiStats)]
        lib.jacobi_csr_destroy.argtypes = [H]
        lib.jacobi_csr_destroy.restype = None
        lib.jacobi_measure_fma_rates.argtypes = [i64, ctypes.POINTER(dbl), ctypes.POINTER(dbl), vp]
        for name in ("jacobi_setup", "jacobi_solve", "jacobi_workspace_size", "jacobi_setup_ex",
                     "jacobi_solve_async", "jacobi_solve_ex", "jacobi_last_stats", "jacobi_residual",
                     "jacobi_get_narrow", "jacobi_last_trace", "jacobi_column_stats", "jacobi_solve_fp64_noalloc",
                     "jacobi_batch_workspace_size", "jacobi_batch_create", "jacobi_batch_solve_async",
                     "jacobi_batch_stats", "jacobi_batch_grid", "jacobi_server_create", "jacobi_server_submit",
                     "jacobi_server_submit_generated", "jacobi_server_step", "jacobi_server_poll",
                     "jacobi_server_rounds", "jacobi_generate_request", "jacobi_csr_setup", "jacobi_csr_solve_async",
                     "jacobi_csr_solve", "jacobi_csr_last_stats", "jacobi_csr_info", "jacobi_csr_last_trace",
                     "jacobi_batch_solve", "jacobi_server_wait", "jacobi_csr_format", "jacobi_measure_fma_rates"):
            getattr(lib, name).restype = i32
        _lib = lib
        return lib


def measure_fma_rates(iters: int = 20000, stream=None) -> tuple[float, float]:
    """FP64 and FP32 FMAs per second of the current device's CUDA cores (``jacobi_measure_fma_rates``)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    f64, f32 = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().jacobi_measure_fma_rates(iters, ctypes.byref(f64), ctypes.byref(f32), s.cuda_stream),
           "jacobi_measure_fma_rates", False)
    return f64.value, f32.value


def _check(status: int, where: str, allow_warn: bool = True) -> int:
    if status < 0 or (status > 0 and not allow_warn):
        raise JacobiError(status, where)
    return status


# ------------------------------------------------------------------------- host-pointer interface

class HostSolver:
    """``jacobi_setup`` / ``jacobi_solve`` with numpy arrays (FP64 path, one right-hand side)."""

    def __init__(self, A: np.ndarray, B: np.ndarray):
        lib = load()
        A = np.ascontiguousarray(A, dtype=np.float64)
        B = np.ascontiguousarray(np.asarray(B, dtype=np.float64).reshape(-1))
        n = A.shape[0]
        if A.shape != (n, n) or B.shape != (n,):
            raise ValueError("A must be (n, n) and B (n,)")
        self.n = n
        self._h = ctypes.c_void_p()
        st = lib.jacobi_setup(A.ctypes.data, B.ctypes.data, n, ctypes.byref(self._h))
        _check(st, "jacobi_setup", allow_warn=False)

    def solve(self, X0=None, max_iter: int = 1000, tol: float = 1e-12):
        """Returns ``(status, X, iters, final_delta)``."""
        lib = load()
        X = np.zeros(self.n)
        x0 = None if X0 is None else np.ascontiguousarray(np.asarray(X0, dtype=np.float64).reshape(-1))
        it = ctypes.c_int64(0)
        de = ctypes.c_double(0.0)
        st = lib.jacobi_solve(self._h, None if x0 is None else x0.ctypes.data, max_iter, tol, X.ctypes.data,
                              ctypes.byref(it), ctypes.byref(de))
        _check(st, "jacobi_solve")
        return st, X, int(it.value), float(de.value)

    def close(self):
        if self._h:
            load().jacobi_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------ device-pointer interface

class DeviceSolver:
    """``jacobi_setup_ex`` / ``jacobi_solve_*`` on CUDA tensors; torch owns the workspace and stream."""

    def __init__(self, A, B, precision: str = "fp64", norm: str = "inf", grid: int = 0, stream=None,
                 copy_a: bool = False, max_outer: int = 0, max_inner: int = 0, inner_rtol: float = 0.0,
                 workspace=None, device=None, split_residual: bool = False, flags: int = 0,
                 method: str = "jacobi", omega: float = 1.0, symmetric: bool = False):
        """A, B: float64 tensors on the GPU (A may be borrowed, see jacobi_desc.A) or on the host (copied
        to the device during setup; pin them for full link bandwidth).  workspace: optional uint8 CUDA
        tensor of at least workspace_size() bytes to reuse across solvers."""
        import torch
        lib = load()
        if A.dtype != torch.float64 or B.dtype != torch.float64:
            raise ValueError("A and B must be float64 tensors")
        if device is None:
            device = A.device if A.is_cuda else torch.device("cuda", torch.cuda.current_device())
        n = A.shape[0]
        if A.dim() != 2 or A.shape[1] != n or A.stride(1) != 1:
            raise ValueError("A must be (n, n) with unit column stride")
        Bv = B.reshape(-1)
        if Bv.numel() != n or Bv.stride(0) != 1:
            raise ValueError("B must hold n contiguous values")
        self.n = n
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        d = JacobiDesc()
        lib.jacobi_desc_init(ctypes.byref(d))
        d.n, d.nrhs = n, 1
        d.precision = PRECISIONS[precision]
        d.norm = NORMS[norm]
        d.A, d.lda = A.data_ptr(), A.stride(0)
        d.B, d.ldb = Bv.data_ptr(), n
        d.stream = self.stream.cuda_stream
        d.grid, d.max_outer, d.max_inner, d.inner_rtol = grid, max_outer, max_inner, inner_rtol
        d.flags = ((FLAG_COPY_A if copy_a else 0) | (FLAG_SPLIT_RESIDUAL if split_residual else 0)
                   | (FLAG_SYMMETRIC if symmetric else 0) | flags)
        d.method = METHODS[method]
        d.omega = omega
        nbytes = ctypes.c_size_t(0)
        with torch.cuda.device(device):
            _check(lib.jacobi_workspace_size(ctypes.byref(d), ctypes.byref(nbytes)), "jacobi_workspace_size")
        if workspace is None or workspace.numel() < nbytes.value:
            workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=device)
        self.workspace = workspace
        d.workspace, d.workspace_bytes = self.workspace.data_ptr(), self.workspace.numel()
        self._A, self._B = A, Bv  # keep the borrowed operands alive
        self._h = ctypes.c_void_p()
        with torch.cuda.device(device):
            _check(lib.jacobi_setup_ex(ctypes.byref(d), ctypes.byref(self._h)), "jacobi_setup_ex", False)
        self.precision = precision

    def solve_async(self, X0=None, max_iter: int = 1000, tol: float = 1e-12, out=None, stats_dev=None):
        """Queue a solve on the solver's stream; returns ``out`` (a float64 CUDA tensor of n values)."""
        import torch
        if out is None:
            out = torch.empty(self.n, dtype=torch.float64, device=self.device)
        x0 = None if X0 is None else X0.reshape(-1)
        if x0 is not None and (x0.dtype != torch.float64 or x0.numel() != self.n or x0.stride(0) != 1):
            raise ValueError("X0 must hold n contiguous float64 values")
        st = load().jacobi_solve_async(self._h, None if x0 is None else x0.data_ptr(), max_iter, tol,
                                       out.data_ptr(), None if stats_dev is None else stats_dev.data_ptr())
        _check(st, "jacobi_solve_async")
        return out

    def last_stats(self) -> JacobiStats:
        st = JacobiStats()
        _check(load().jacobi_last_stats(self._h, ctypes.byref(st)), "jacobi_last_stats")
        return st

    def solve(self, X0=None, max_iter: int = 1000, tol: float = 1e-12, out=None):
        """Synchronous solve: returns ``(X, stats)``; raises on error statuses (< 0)."""
        out = self.solve_async(X0, max_iter, tol, out)
        st = self.last_stats()
        _check(st.status, "solve")
        return out, st

    def narrow(self):
        """Host copy of the narrow off-diagonal matrix the inner sweeps read, as raw codes
        (float32 / uint16 BF16 codes / uint8 E4M3 codes, shape (n, n)), and the E4M3 row scales."""
        dt = {"fp32_ir": np.float32, "bf16_ir": np.uint16, "fp8_ir": np.uint8}[self.precision]
        out = np.zeros((self.n, self.n), dtype=dt)
        scale = np.zeros(self.n, dtype=np.float32)
        _check(load().jacobi_get_narrow(self._h, out.ctypes.data, self.n, scale.ctypes.data), "jacobi_get_narrow")
        return out, scale

    def trace(self):
        """Device-side phase trace of the last solve: list of (kind, start_ns, end_ns) per phase."""
        cap = 512
        t = np.zeros(cap, dtype=np.int64)
        k = np.zeros(cap, dtype=np.int32)
        cnt = ctypes.c_int32(0)
        _check(load().jacobi_last_trace(self._h, t.ctypes.data, k.ctypes.data, cap, ctypes.byref(cnt)),
               "jacobi_last_trace")
        m = min(cap, cnt.value)
        out, prev = [], 0
        for i in range(m):
            out.append((int(k[i]), prev, int(t[i])))
            prev = int(t[i])
        return out

    def residual(self, X) -> float:
        """||B - A X||_inf / ||B||_inf on the device in FP64."""
        rel = ctypes.c_double(0.0)
        _check(load().jacobi_residual(self._h, X.data_ptr(), ctypes.byref(rel)), "jacobi_residual")
        return float(rel.value)

    def close(self):
        if self._h:
            load().jacobi_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



# ------------------------------------------------------------------------------- sparse interface

class CsrSolver:
    """``jacobi_csr_*``: Jacobi for a sparse A in CSR (int64 row offsets, int32 columns strictly ascending in
    each row with the diagonal stored, float64 values) and one right-hand side; precision "fp64" (the plain
    iteration) or "fp32_ir" / "bf16_ir" (mixed-precision refinement to a relative residual).  The arrays may be torch
    tensors on the GPU or the host, or numpy arrays; setup copies them into the library's layout (DIA for a
    matrix whose entries lie on a few diagonals, else sliced ELL; ``flags=FLAG_CSR_ELL`` forces ELL), so
    they may be dropped afterwards."""

    def __init__(self, row_ptr, col_idx, values, B, norm: str = "inf", flags: int = 0, stream=None, device=None,
                 precision: str = "fp64", inner_rtol: float = 0.0, max_inner: int = 0, max_outer: int = 0):
        import torch
        lib = load()

        def as_tensor(a, dtype):
            t = torch.as_tensor(a)
            if t.dtype != dtype:
                raise ValueError(f"expected {dtype}, got {t.dtype}")
            return t.contiguous()

        rp = as_tensor(row_ptr, torch.int64)
        ci = as_tensor(col_idx, torch.int32)
        va = as_tensor(values, torch.float64)
        b = as_tensor(B, torch.float64).reshape(-1)
        self.n = rp.numel() - 1
        if b.numel() != self.n or ci.numel() != va.numel():
            raise ValueError("CSR shape mismatch")
        if device is None:
            device = va.device if va.is_cuda else torch.device("cuda", torch.cuda.current_device())
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        d = JacobiCsrDesc()
        d.n, d.nnz = self.n, ci.numel()
        d.row_ptr, d.col_idx, d.values, d.B = rp.data_ptr(), ci.data_ptr(), va.data_ptr(), b.data_ptr()
        d.norm, d.flags, d.stream = NORMS[norm], flags, self.stream.cuda_stream
        d.precision = PRECISIONS[precision]
        d.max_outer, d.max_inner, d.inner_rtol = max_outer, max_inner, inner_rtol
        self.precision = precision
        self._h = ctypes.c_void_p()
        with torch.cuda.device(device):
            _check(lib.jacobi_csr_setup(ctypes.byref(d), ctypes.byref(self._h)), "jacobi_csr_setup", False)

    def solve_async(self, X0=None, max_iter: int = 1000, tol: float = 1e-12, out=None):
        """Queue a solve on the solver's stream; returns ``out`` (n float64 values on the GPU)."""
        import torch
        if out is None:
            out = torch.empty(self.n, dtype=torch.float64, device=self.device)
        x0 = None if X0 is None else torch.as_tensor(X0).reshape(-1)
        if x0 is not None and (x0.dtype != torch.float64 or x0.numel() != self.n or not x0.is_contiguous()):
            raise ValueError("X0 must hold n contiguous float64 values")
        self._x0 = x0  # alive until the copy is queued
        _check(load().jacobi_csr_solve_async(self._h, None if x0 is None else x0.data_ptr(), max_iter, tol,
                                             out.data_ptr()), "jacobi_csr_solve_async")
        return out

    def last_stats(self) -> JacobiStats:
        st = JacobiStats()
        _check(load().jacobi_csr_last_stats(self._h, ctypes.byref(st)), "jacobi_csr_last_stats")
        return st

    def solve(self, X0=None, max_iter: int = 1000, tol: float = 1e-12, out=None):
        """Synchronous solve: returns ``(X, stats)``; raises on error statuses (< 0)."""
        out = self.solve_async(X0, max_iter, tol, out)
        st = self.last_stats()
        _check(st.status, "solve")
        return out, st

    def info(self) -> dict:
        stored, slices, grid = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int32(0)
        _check(load().jacobi_csr_info(self._h, ctypes.byref(stored), ctypes.byref(slices), ctypes.byref(grid)),
               "jacobi_csr_info")
        fmt, ndiag = ctypes.c_int32(0), ctypes.c_int32(0)
        _check(load().jacobi_csr_format(self._h, ctypes.byref(fmt), ctypes.byref(ndiag)), "jacobi_csr_format")
        return {"stored_slots": stored.value, "slices": slices.value, "grid": grid.value,
                "format": "dia" if fmt.value == 1 else "ell", "diagonals": ndiag.value}

    def trace(self):
        """Device-side end time of every phase of the last solve: list of (start_ns, end_ns)."""
        t, _ = self._trace()
        return [(int(t[i - 1]) if i else 0, int(t[i])) for i in range(len(t))]

    def kinds(self):
        """Kind (JACOBI_PHASE_*) of every phase of the last solve, in the order of trace()."""
        return [int(k) for k in self._trace()[1]]

    def _trace(self):
        cap = 512
        t = np.zeros(cap, dtype=np.int64)
        k = np.zeros(cap, dtype=np.int32)
        cnt = ctypes.c_int32(0)
        _check(load().jacobi_csr_last_trace(self._h, t.ctypes.data, k.ctypes.data, cap, ctypes.byref(cnt)),
               "jacobi_csr_last_trace")
        m = min(cap, cnt.value)
        return t[:m], k[:m]

    def close(self):
        if self._h:
            load().jacobi_csr_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------------ batched interface

class BatchSolver:
    """``jacobi_batch_*``: many independent systems (lists of float64 CUDA tensors), one persistent
    kernel per solve, replayed from a captured CUDA graph."""

    def __init__(self, As, Bs, precision: str = "fp32_ir", rows_per_warp: int = 0, ctas_per_sm: int = 0,
                 max_outer: int = 0, max_inner: int = 0, inner_rtol: float = 0.0, stream=None, workspace=None,
                 split_residual: bool = False):
        import torch
        lib = load()
        if len(As) != len(Bs) or not As:
            raise ValueError("need one B per A")
        self.count = len(As)
        self.device = As[0].device
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._A = [a.contiguous() for a in As]
        self._B = [b.reshape(-1).contiguous() for b in Bs]
        for a, b in zip(self._A, self._B):
            if a.dtype != torch.float64 or b.dtype != torch.float64 or not a.is_cuda or a.shape[0] != b.numel():
                raise ValueError("A_k (n_k x n_k) and B_k (n_k) must be float64 CUDA tensors")
        self.n = np.array([a.shape[0] for a in self._A], dtype=np.int64)
        self.X = [torch.zeros(int(k), dtype=torch.float64, device=self.device) for k in self.n]
        self._pa = (ctypes.c_void_p * self.count)(*[a.data_ptr() for a in self._A])
        self._pb = (ctypes.c_void_p * self.count)(*[b.data_ptr() for b in self._B])
        self._px = (ctypes.c_void_p * self.count)(*[x.data_ptr() for x in self.X])
        d = JacobiBatchDesc()
        d.count = self.count
        d.n = self.n.ctypes.data
        d.A, d.B, d.X = ctypes.addressof(self._pa), ctypes.addressof(self._pb), ctypes.addressof(self._px)
        d.precision = PRECISIONS[precision]
        d.rows_per_warp, d.ctas_per_sm = rows_per_warp, ctas_per_sm
        d.max_outer, d.max_inner, d.inner_rtol = max_outer, max_inner, inner_rtol
        d.flags = FLAG_SPLIT_RESIDUAL if split_residual else 0
        d.stream = self.stream.cuda_stream
        nbytes = ctypes.c_size_t(0)
        _check(lib.jacobi_batch_workspace_size(ctypes.byref(d), ctypes.byref(nbytes)), "jacobi_batch_workspace_size")
        if workspace is None or workspace.numel() < nbytes.value:
            workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        self.workspace = workspace
        d.workspace, d.workspace_bytes = workspace.data_ptr(), workspace.numel()
        self._desc = d
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.jacobi_batch_create(ctypes.byref(d), ctypes.byref(self._h)), "jacobi_batch_create", False)
        self.grid = lib.jacobi_batch_grid(self._h)

    def solve_async(self, max_iter: int = 5000, tol: float = 1e-10):
        _check(load().jacobi_batch_solve_async(self._h, max_iter, tol), "jacobi_batch_solve_async")
        return self.X

    def stats(self):
        arr = (JacobiStats * self.count)()
        _check(load().jacobi_batch_stats(self._h, ctypes.addressof(arr)), "jacobi_batch_stats")
        return list(arr)

    def close(self):
        if self._h:
            load().jacobi_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MultiSolver:
    """Many right-hand sides through ``jacobi_setup_ex`` (nrhs = r) / ``jacobi_solve_ex``: plain FP64
    Jacobi, or BF16 inner sweeps on tcgen05 tensor cores with FP64 refinement.  B and X are (r, n)
    float64 CUDA tensors (row c is right-hand side c, i.e. column-major n x r)."""

    def __init__(self, A, B, precision: str = "bf16_ir", stream=None, max_outer: int = 0, max_inner: int = 0,
                 inner_rtol: float = 0.0, norm: str = "inf", split_residual: bool = False,
                 retire_columns: bool = False, tc_residual: bool = False, flags: int = 0):
        import torch
        lib = load()
        n = A.shape[0]
        if B.dim() != 2 or B.shape[1] != n or B.stride(1) != 1:
            raise ValueError("B must be (r, n) with unit stride along n")
        self.n, self.r = n, B.shape[0]
        self.device = A.device
        self.stream = stream if stream is not None else torch.cuda.current_stream(A.device)
        d = JacobiDesc()
        lib.jacobi_desc_init(ctypes.byref(d))
        d.n, d.nrhs = n, self.r
        d.precision = PRECISIONS[precision]
        d.norm = NORMS[norm]
        d.A, d.lda = A.data_ptr(), A.stride(0)
        d.B, d.ldb = B.data_ptr(), B.stride(0)
        d.stream = self.stream.cuda_stream
        d.max_outer, d.max_inner, d.inner_rtol = max_outer, max_inner, inner_rtol
        d.flags = ((FLAG_SPLIT_RESIDUAL if split_residual else 0) | (FLAG_RETIRE_COLUMNS if retire_columns else 0)
                   | (FLAG_TC_RESIDUAL if tc_residual else 0) | flags)
        nbytes = ctypes.c_size_t(0)
        with torch.cuda.device(A.device):
            _check(lib.jacobi_workspace_size(ctypes.byref(d), ctypes.byref(nbytes)), "jacobi_workspace_size")
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=A.device)
        d.workspace, d.workspace_bytes = self.workspace.data_ptr(), self.workspace.numel()
        self._A, self._B = A, B
        self._h = ctypes.c_void_p()
        with torch.cuda.device(A.device):
            _check(lib.jacobi_setup_ex(ctypes.byref(d), ctypes.byref(self._h)), "jacobi_setup_ex", False)

    def trace(self):
        """Per-phase CUDA-event timeline of the last solve: list of (kind, start_ns, end_ns)."""
        return DeviceSolver.trace(self)

    def column_stats(self):
        """Per column of the last solve: (iterations after which it finished, its last change norm or
        relative residual), as numpy arrays."""
        iters = np.zeros(self.r, dtype=np.int64)
        vals = np.zeros(self.r, dtype=np.float64)
        _check(load().jacobi_column_stats(self._h, iters.ctypes.data, vals.ctypes.data), "jacobi_column_stats")
        return iters, vals

    def solve(self, X0=None, max_iter: int = 5000, tol: float = 1e-10, out=None):
        """Returns ``(X, stats)`` with X an (r, n) tensor; raises on error statuses (< 0)."""
        import torch
        if out is None:
            out = torch.empty(self.r, self.n, dtype=torch.float64, device=self.device)
        st = JacobiStats()
        rc = load().jacobi_solve_ex(self._h, None if X0 is None else X0.data_ptr(), max_iter, tol, out.data_ptr(),
                                    ctypes.byref(st))
        _check(rc, "jacobi_solve_ex")
        return out, st

    def close(self):
        if self._h:
            load().jacobi_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_solve(As, Bs, Xs, tol: float = 1e-10, max_iter: int = 5000, precision: str = "fp32_ir"):
    """``jacobi_batch_solve``: one call for a batch (lists of float64 CUDA tensors A_k (n_k, n_k), B_k and
    outputs X_k (n_k,)).  Returns (worst status, per-system records)."""
    lib = load()
    count = len(As)
    ns = np.array([a.shape[0] for a in As], dtype=np.int64)
    pa = (ctypes.c_void_p * count)(*[a.data_ptr() for a in As])
    pb = (ctypes.c_void_p * count)(*[b.data_ptr() for b in Bs])
    px = (ctypes.c_void_p * count)(*[x.data_ptr() for x in Xs])
    sts = (JacobiStats * count)()
    st = lib.jacobi_batch_solve(count, ns.ctypes.data, ctypes.addressof(pa), ctypes.addressof(pb),
                                ctypes.addressof(px), tol, max_iter, PRECISIONS[precision], ctypes.addressof(sts))
    _check(st, "jacobi_batch_solve")
    return st, [sts[k] for k in range(count)]


# ------------------------------------------------------------------------------ serving interface

def generate_request(n: int, r: int, f: float, seed: int, device=None, stream=None):
    """A (n, n) and B (r, n) float64 CUDA tensors of the seeded serving generator (bit-identical to
    ``synth.serving_request``)."""
    import torch
    device = device or torch.device("cuda", torch.cuda.current_device())
    stream = stream if stream is not None else torch.cuda.current_stream(device)
    A = torch.empty(n, n, dtype=torch.float64, device=device)
    B = torch.zeros(r, n, dtype=torch.float64, device=device)
    _check(load().jacobi_generate_request(n, r, f, seed, A.data_ptr(), B.data_ptr(), n, stream.cuda_stream),
           "jacobi_generate_request")
    return A, B


class Server:
    """``jacobi_server_*``: continuous batching of independent requests (see include/jacobi.h)."""

    def __init__(self, budget_bytes: int, tol: float = 1e-10, max_active: int = 0, inner_rtol: float = 0.0,
                 max_inner: int = 0, max_outer: int = 0, stream=None, split_residual: bool = False,
                 tc_residual: bool = False):
        import torch
        lib = load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        d = JacobiServerDesc()
        d.budget_bytes, d.tol, d.max_active = budget_bytes, tol, max_active
        d.flags = (FLAG_SPLIT_RESIDUAL if split_residual else 0) | (FLAG_TC_RESIDUAL if tc_residual else 0)
        d.inner_rtol, d.max_inner, d.max_outer = inner_rtol, max_inner, max_outer
        d.stream = self.stream.cuda_stream
        self._h = ctypes.c_void_p()
        _check(lib.jacobi_server_create(ctypes.byref(d), ctypes.byref(self._h)), "jacobi_server_create", False)
        self._keep = {}

    def submit_generated(self, n: int, r: int, f: float, seed: int, out) -> int:
        rid = ctypes.c_int64(0)
        _check(load().jacobi_server_submit_generated(self._h, n, r, f, seed, out.data_ptr(), ctypes.byref(rid)),
               "jacobi_server_submit_generated")
        self._keep[rid.value] = out
        return rid.value

    def submit(self, A, B, out) -> int:
        """A (n, n), B (r, n) float64 tensors (device or host); out (r, n) receives X."""
        rid = ctypes.c_int64(0)
        _check(load().jacobi_server_submit(self._h, A.shape[0], B.shape[0], A.data_ptr(), B.data_ptr(),
                                           out.data_ptr(), ctypes.byref(rid)), "jacobi_server_submit")
        self._keep[rid.value] = (A, B, out)
        return rid.value

    def step(self):
        a, p = ctypes.c_int32(0), ctypes.c_int32(0)
        _check(load().jacobi_server_step(self._h, ctypes.byref(a), ctypes.byref(p)), "jacobi_server_step")
        return a.value, p.value

    def poll(self, cap: int = 4096):
        ids = np.zeros(cap, dtype=np.int64)
        sts = (JacobiStats * cap)()
        cnt = ctypes.c_int32(0)
        _check(load().jacobi_server_poll(self._h, ids.ctypes.data, ctypes.addressof(sts), cap, ctypes.byref(cnt)),
               "jacobi_server_poll")
        out = [(int(ids[i]), sts[i]) for i in range(cnt.value)]
        for rid, _ in out:
            self._keep.pop(rid, None)
        return out

    def wait(self, rid: int) -> JacobiStats:
        """Run rounds until request ``rid`` finishes; returns its record (the request is collected)."""
        st = JacobiStats()
        _check(load().jacobi_server_wait(self._h, rid, ctypes.byref(st)), "jacobi_server_wait")
        self._keep.pop(rid, None)
        return st

    def rounds(self) -> int:
        r = ctypes.c_int64(0)
        _check(load().jacobi_server_rounds(self._h, ctypes.byref(r)), "jacobi_server_rounds")
        return r.value

    def close(self):
        if self._h:
            load().jacobi_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
