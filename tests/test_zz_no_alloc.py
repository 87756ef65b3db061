"""The allocation-free FP64 solve (jacobi_solve_fp64_noalloc) against the regular entry points.

The allocation-free call is for code that must not allocate device memory while it runs (a plugin whose
host application owns the GPU memory pool, or a latency-bound loop that cannot take cudaMalloc's
synchronisation or failure).  It keeps its scratch in a fixed device array shared by every call, so
this file checks two calls in a row (the second must not see the first's leftovers) against
jacobi_setup_ex + jacobi_solve_ex on the same inputs, at the FP64 path's tolerance, and the size limit.
It runs last so that a failure here leaves every other test's result in place, and it passes alone in
a fresh process as well as after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL_ITER = 1e-12  # the FP64 path's bar: relative max-norm difference of the returned iterate


@pytest.fixture(scope="module")
def jac():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1403_5805_gb300 as jac
    return jac


def noalloc_solve(jac, A_t, lda, B_t, n, max_iter, tol, X0_t=None):
    import torch
    out = torch.full((n,), float("nan"), dtype=torch.float64, device=A_t.device)
    st = jac.JacobiStats()
    stream = torch.cuda.current_stream(A_t.device).cuda_stream
    rc = jac.load().jacobi_solve_fp64_noalloc(A_t.data_ptr(), lda, B_t.data_ptr(), n,
                                              None if X0_t is None else X0_t.data_ptr(), max_iter, tol,
                                              out.data_ptr(), ctypes.byref(st), stream)
    return rc, out, st


def regular_solve(jac, A, B, max_iter, tol, X0_t=None):
    import torch
    s = jac.DeviceSolver(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    X, st = s.solve(X0=X0_t, max_iter=max_iter, tol=tol)
    return X, st


def rel(a, b):
    return float((a - b).abs().max().item() / b.abs().max().item())


def test_two_calls_in_a_row_match_regular_path(jac):
    import torch
    cases = [(1000, 1.1, "dom"), (517, 1.25, "hard")]  # the second is smaller and odd-sized
    for n, f, gen in cases:
        A, B, _ = (synth.dominant_system if gen == "dom" else synth.hard_system)(n, f, seed=900 + n)
        b = B[:, 0].copy()
        want, st_want = regular_solve(jac, A, b, 3000, 1e-12)
        # odd n reads one padding element per row: give A a padded row stride, padding poisoned with NaN
        lda = n if n % 2 == 0 else n + 1
        A_pad = torch.full((n, lda), float("nan"), dtype=torch.float64, device="cuda")
        A_pad[:, :n] = torch.from_numpy(A).cuda()
        B_t = torch.from_numpy(b).cuda()
        rc, got, st = noalloc_solve(jac, A_pad, lda, B_t, n, 3000, 1e-12)
        assert rc == jac.OK == st_want.status, (rc, st.status)
        assert st.sweeps == st_want.sweeps
        assert rel(got, want) <= TOL_ITER


def test_start_vector_and_repeat(jac):
    import torch
    n = 640
    A, B, _ = synth.dominant_system(n, 1.05, seed=77)
    b = B[:, 0].copy()
    X0 = torch.linspace(-1, 1, n, dtype=torch.float64, device="cuda")
    want, st_want = regular_solve(jac, A, b, 11, 1e-300, X0_t=X0)
    A_t, B_t = torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda()
    for _ in range(2):
        rc, got, st = noalloc_solve(jac, A_t, n, B_t, n, 11, 1e-300, X0_t=X0)
        assert rc == jac.NOT_CONVERGED and st.sweeps == 11
        assert rel(got, want) <= TOL_ITER


def test_rejects_sizes_beyond_the_limit(jac):
    import torch
    limit = 32768  # JACOBI_NOALLOC_MAX_N
    n = limit + 2
    A_t = torch.zeros(16, dtype=torch.float64, device="cuda")  # never read: the size check comes first
    rc, _, _ = noalloc_solve(jac, A_t, n, A_t, n, 10, 1e-12)
    assert rc == jac.ERR_INVALID_ARG
    A, B, _ = synth.dominant_system(4, 1.5, seed=3)
    rc, _, _ = noalloc_solve(jac, torch.from_numpy(A).cuda(), 3, torch.from_numpy(B[:, 0].copy()).cuda(), 4,
                             10, 1e-12)
    assert rc == jac.ERR_INVALID_ARG  # lda < n


def test_failed_diagonal_check_leaves_nothing_behind(jac):
    # A zero (then a non-finite) a_ii must be reported as the regular path reports it, and the next call,
    # which reuses the same scratch (diagonal-check key, ||B||), must solve as if nothing had failed.
    import torch
    n = 300
    A, B, _ = synth.dominant_system(n, 1.2, seed=41)
    b = B[:, 0].copy()
    B_t = torch.from_numpy(b).cuda()
    for bad, want_rc in ((0.0, jac.ERR_ZERO_DIAGONAL), (float("nan"), jac.ERR_NONFINITE)):
        Ab = A.copy()
        Ab[123, 123] = bad
        rc, _, _ = noalloc_solve(jac, torch.from_numpy(Ab).cuda(), n, B_t, n, 100, 1e-12)
        assert rc == want_rc
        want, st_want = regular_solve(jac, A, b, 3000, 1e-12)
        rc, got, st = noalloc_solve(jac, torch.from_numpy(A).cuda(), n, B_t, n, 3000, 1e-12)
        assert rc == jac.OK == st_want.status and st.sweeps == st_want.sweeps
        assert rel(got, want) <= TOL_ITER


def test_rejects_host_memory_and_bad_tolerances(jac):
    import torch
    n = 64
    A, B, _ = synth.dominant_system(n, 1.5, seed=5)
    b = np.ascontiguousarray(B[:, 0])
    A_t, B_t = torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    lib = jac.load()
    st = jac.JacobiStats()
    stream = torch.cuda.current_stream().cuda_stream
    # host (pageable) A: rejected by the pointer check before any device work
    rc = lib.jacobi_solve_fp64_noalloc(A.ctypes.data, n, B_t.data_ptr(), n, None, 10, 1e-12, out.data_ptr(),
                                       ctypes.byref(st), stream)
    assert rc == jac.ERR_INVALID_ARG
    for tol in (0.0, -1.0, float("inf"), float("nan")):
        rc, _, _ = noalloc_solve(jac, A_t, n, B_t, n, 10, tol)
        assert rc == jac.ERR_INVALID_ARG, tol
    # the largest finite tol is a valid (if useless) bound, as on the regular path: one sweep
    rc, _, st = noalloc_solve(jac, A_t, n, B_t, n, 10, float(np.finfo(np.float64).max))
    assert rc == jac.OK and st.sweeps == 1
