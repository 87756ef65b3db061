"""FP64 path on the GPU against the CPU oracle, through the C ABI.

The bar (Section 2 iteration, same inputs on both sides): every iterate X^(k) within 1e-12 relative
max-norm of the oracle's, and the sweep count and status exactly equal.
"""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_ITER = 1e-12


@pytest.fixture(scope="module")
def jac():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1403_5805_gb300 as jac
    return jac


def dev_solver(jac, A, B, **kw):
    import torch
    At = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    Bt = torch.from_numpy(np.ascontiguousarray(B).reshape(-1)).cuda()
    return jac.DeviceSolver(At, Bt, **kw)


def rel_err(x, ref):
    return float(np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300))


def make(gen, n, f, seed):
    return (synth.dominant_system if gen == "dom" else synth.hard_system)(n, f, seed)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 33, 100, 127, 257, 512, 1000, 1537])
@pytest.mark.parametrize("gen", ["dom", "hard"])
def test_every_iterate_matches_oracle(jac, n, gen):
    A, B, _ = make(gen, n, 1.25, seed=1000 + n)
    K = 10
    ref = oracle.jacobi(A, B, max_iter=K, tol=1e-300, trace=True)
    s = dev_solver(jac, A, B)
    for k in range(1, ref.iters + 1):
        X, st = s.solve(max_iter=k, tol=1e-300)
        assert st.sweeps == k
        assert st.status == (jac.OK if (k == ref.iters and ref.status == 0) else jac.NOT_CONVERGED)
        err = rel_err(X.cpu().numpy(), ref.trace[k - 1][:, 0])
        assert err <= TOL_ITER, (k, err)


@pytest.mark.parametrize("gen,n,f", [("dom", 64, 1.25), ("dom", 512, 1.25), ("dom", 2048, 1.05),
                                     ("hard", 256, 1.25), ("hard", 1000, 1.05), ("hard", 4097, 1.1)])
def test_converged_solve_matches_oracle(jac, gen, n, f):
    A, B, Xs = make(gen, n, f, seed=7 + n)
    tol = 1e-12
    ref = oracle.jacobi(A, B, max_iter=5000, tol=tol, nthreads=os.cpu_count() or 1)
    s = dev_solver(jac, A, B)
    X, st = s.solve(max_iter=5000, tol=tol)
    assert ref.status == 0 and st.status == 0
    assert st.sweeps == ref.iters
    assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= TOL_ITER
    # the change is a difference of O(||X||) numbers: its rounding error is absolute, at the iterate level
    assert abs(st.final_delta - ref.delta) <= 2 * TOL_ITER * np.max(np.abs(ref.X))


def test_paper_config_n512(jac):
    """n = 512, f = 1.25, X0 = 0, tol 1e-12 on max|dX|, max_iter 2000."""
    A, B, Xs = synth.dominant_system(512, 1.25, seed=synth.BASE_SEED)
    ref = oracle.jacobi(A, B, max_iter=2000, tol=1e-12)
    s = dev_solver(jac, A, B)
    X, st = s.solve(max_iter=2000, tol=1e-12)
    assert (st.status, st.sweeps) == (ref.status, ref.iters)
    assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= TOL_ITER
    assert np.max(np.abs(X.cpu().numpy() - Xs[:, 0])) <= 1e-11


def test_full_size_single_system(jac):
    """n = 16384, f = 1.05: all n outputs against the oracle (run on all host cores)."""
    A, B, _ = synth.dominant_system(16384, 1.05, seed=synth.BASE_SEED + 1)
    ref = oracle.jacobi(A, B, max_iter=2000, tol=1e-12, nthreads=os.cpu_count() or 1)
    s = dev_solver(jac, A, B)
    X, st = s.solve(max_iter=2000, tol=1e-12)
    assert (st.status, st.sweeps) == (ref.status, ref.iters)
    assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= TOL_ITER


@pytest.mark.parametrize("norm,onorm", [("2", oracle.NORM_2), ("resid", oracle.NORM_RESID)])
def test_other_stopping_norms(jac, norm, onorm):
    A, B, _ = synth.hard_system(700, 1.25, seed=5)
    tol = 1e-9
    ref = oracle.jacobi(A, B, max_iter=1000, tol=tol, norm=onorm)
    s = dev_solver(jac, A, B, norm=norm)
    X, st = s.solve(max_iter=1000, tol=tol)
    assert (st.status, st.sweeps) == (ref.status, ref.iters)
    # absolute rounding bound of the change norm, from the iterate tolerance
    xs = np.max(np.abs(ref.X))
    scale = np.sqrt(A.shape[0]) * xs if norm == "2" else np.max(np.abs(np.diag(A))) * xs / np.max(np.abs(B))
    assert abs(st.final_delta - ref.delta) <= 2 * TOL_ITER * scale
    assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= TOL_ITER


def test_start_vector_and_cap(jac):
    A, B, _ = synth.hard_system(300, 1.05, seed=3)
    X0 = np.linspace(-1, 1, 300)
    ref = oracle.jacobi(A, B, X0=X0, max_iter=17, tol=1e-14)
    s = dev_solver(jac, A, B)
    import torch
    X, st = s.solve(X0=torch.from_numpy(X0).cuda(), max_iter=17, tol=1e-14)
    assert st.status == jac.NOT_CONVERGED == ref.status and st.sweeps == 17
    assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= TOL_ITER


def test_resume_is_bitwise(jac):
    """Jacobi is memoryless: a solve split in two equals the whole solve bit for bit."""
    import torch
    A, B, _ = synth.hard_system(900, 1.1, seed=11)
    s = dev_solver(jac, A, B)
    whole, _ = s.solve(max_iter=30, tol=1e-300)
    half, _ = s.solve(max_iter=12, tol=1e-300)
    rest, _ = s.solve(X0=half.clone(), max_iter=18, tol=1e-300)
    assert torch.equal(whole, rest)


def test_deterministic_and_grid_independent(jac):
    import torch
    A, B, _ = synth.dominant_system(1000, 1.1, seed=12)
    ref = oracle.jacobi(A, B, max_iter=8, tol=1e-300)
    outs = {}
    for g in (1, 7, 0):
        s = dev_solver(jac, A, B, grid=g)
        a, _ = s.solve(max_iter=8, tol=1e-300)
        b, _ = s.solve(max_iter=8, tol=1e-300)
        assert torch.equal(a, b)
        assert rel_err(a.cpu().numpy(), ref.X[:, 0]) <= TOL_ITER
        outs[g] = a
    # the dot-product order depends on the chunking, not on the grid: identical across grids
    assert torch.equal(outs[1], outs[7]) and torch.equal(outs[1], outs[0])


def test_borrowed_and_copied_A_agree(jac):
    import torch
    A, B, _ = synth.dominant_system(1024, 1.25, seed=13)
    a, _ = dev_solver(jac, A, B).solve(max_iter=6, tol=1e-300)
    b, _ = dev_solver(jac, A, B, copy_a=True).solve(max_iter=6, tol=1e-300)
    assert torch.equal(a, b)


def test_strided_A_view(jac):
    import torch
    n = 301
    A, B, _ = synth.dominant_system(n, 1.25, seed=14)
    big = torch.zeros(n, n + 7, dtype=torch.float64, device="cuda")
    big[:, :n] = torch.from_numpy(A).cuda()
    ref = oracle.jacobi(A, B, max_iter=9, tol=1e-300)
    s = jac.DeviceSolver(big[:, :n], torch.from_numpy(B[:, 0].copy()).cuda())
    X, st = s.solve(max_iter=9, tol=1e-300)
    assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= TOL_ITER


def test_host_pointer_interface(jac):
    A, B, _ = synth.dominant_system(200, 1.25, seed=15)
    ref = oracle.jacobi(A, B, max_iter=100, tol=1e-12)
    h = jac.HostSolver(A, B[:, 0])
    st, X, iters, delta = h.solve(max_iter=100, tol=1e-12)
    assert (st, iters) == (ref.status, ref.iters)
    assert rel_err(X, ref.X[:, 0]) <= TOL_ITER
    h.close()


def test_diagonal_matrix_one_sweep(jac):
    d = np.array([2.0, -3.0, 7.0, 0.1, 1e3, 5.0])
    A = np.diag(d)
    B = np.array([1.0, 1.0, -2.0, 5.0, 3.0, -1.0])
    s = dev_solver(jac, A, B)
    X, st = s.solve(max_iter=10, tol=1e-12)
    # T = 0, so X^1 = C = D^-1 B; the kernel applies D^-1 as the rounded reciprocal, the oracle divides:
    # within one rounding of each other, and the second sweep changes nothing
    np.testing.assert_allclose(X.cpu().numpy(), B / d, rtol=2.3e-16, atol=0)
    assert st.sweeps == 2 and st.final_delta == 0.0


def test_error_statuses(jac):
    A = np.array([[1.0, 0.1], [0.2, 0.0]])
    with pytest.raises(jac.JacobiError) as e:
        dev_solver(jac, A, np.ones(2))
    assert e.value.status == jac.ERR_ZERO_DIAGONAL
    A[1, 1] = np.nan
    with pytest.raises(jac.JacobiError) as e:
        dev_solver(jac, A, np.ones(2))
    assert e.value.status == jac.ERR_NONFINITE
    # zero diagonal in a later row than a non-finite one: the first failing row decides, as in the oracle
    A = np.eye(5)
    A[1, 1] = 0.0
    A[3, 3] = np.inf
    with pytest.raises(jac.JacobiError) as e:
        dev_solver(jac, A, np.ones(5))
    assert e.value.status == oracle.jacobi(A, np.ones(5)).status == jac.ERR_ZERO_DIAGONAL
    s = dev_solver(jac, np.eye(3), np.ones(3))
    with pytest.raises(jac.JacobiError) as e:
        s.solve(max_iter=0)
    assert e.value.status == jac.ERR_INVALID_ARG
    with pytest.raises(jac.JacobiError):
        s.solve(max_iter=5, tol=0.0)


def test_divergence_reports_nonfinite(jac):
    A = np.array([[1.0, 10.0], [10.0, 1.0]])
    ref = oracle.jacobi(A, np.ones(2), max_iter=2000, tol=1e-12)
    s = dev_solver(jac, A, np.ones(2))
    with pytest.raises(jac.JacobiError) as e:
        s.solve(max_iter=2000, tol=1e-12)
    assert e.value.status == jac.ERR_NONFINITE == ref.status
    assert s.last_stats().sweeps == ref.iters


@pytest.mark.parametrize("prec", ["fp64", "bf16_ir"])
def test_bounded_wait_expires_and_context_stays_usable(jac, prec):
    """Failure detection without a GPU fault: the first ring item of the solve is announced but never
    copied, so the consumers' bounded wait (50 ms here) runs out; the kernel reports a timeout, drains its
    copies and returns, and the next solve on the same context is correct."""
    A, B, _ = synth.dominant_system(2048, 1.25, seed=3)
    flags = jac.binding.FLAG_SHORT_WAITS | jac.binding.FLAG_TEST_DROP_COPY
    bad = dev_solver(jac, A, B, precision=prec, flags=flags)
    with pytest.raises(jac.JacobiError) as e:
        bad.solve(max_iter=50, tol=1e-12 if prec == "fp64" else 1e-10)
    assert e.value.status == jac.ERR_TIMEOUT
    good = dev_solver(jac, A, B, precision=prec)
    X, st = good.solve(max_iter=500, tol=1e-12 if prec == "fp64" else 1e-10)
    assert st.status == 0
    if prec == "fp64":
        ref = oracle.jacobi(A, B, max_iter=500, tol=1e-12)
        assert st.sweeps == ref.iters and rel_err(X.cpu().numpy(), ref.X[:, 0]) <= TOL_ITER
    else:
        _, rel = oracle.residual(A, B, X.cpu().numpy())
        assert rel <= 1e-10


def test_measured_fma_rates_are_plausible(jac):
    # the measurement behind the FP64-FMA bound of the FP64 passes: GB300's CUDA cores issue FP64 FMAs at a
    # small fraction of their FP32 rate (nominally about 1.2 TFLOP/s FP64 against tens of TFLOP/s FP32)
    f64, f32 = jac.measure_fma_rates(iters=20000)
    assert 1e11 < f64 < 1e13, f64
    assert f32 > 8 * f64, (f32, f64)
