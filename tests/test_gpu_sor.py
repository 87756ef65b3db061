"""Gauss-Seidel / SOR (JACOBI_METHOD_SOR) on the GPU against the CPU oracle's sequential sweep.

The GPU runs the sweep as a chain over its CTAs' row blocks; its iterates must be those of the oracle's
block_sor with one block (classical Gauss-Seidel / SOR): within 1e-12 (relative max-norm) after 1, 2
and 5 sweeps, and the same sweep count to convergence, for any grid.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jac():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1403_5805_gb300 as jac
    return jac


def solver(jac, A, B, **kw):
    import torch
    At = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    Bt = torch.from_numpy(np.ascontiguousarray(B[:, 0])).cuda()
    return jac.DeviceSolver(At, Bt, precision="fp64", method="sor", **kw)


def rel_err(x, ref):
    return np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300)


@pytest.mark.parametrize("n,gen,f,omega", [(1, "dom", 1.2, 1.0), (37, "dom", 1.2, 1.0), (300, "hard", 1.1, 1.0),
                                           (1000, "dom", 1.05, 0.8), (777, "dom", 1.2, 1.2),
                                           (2000, "hard", 1.05, 1.0)])
def test_sor_iterates_match_the_sequential_oracle(jac, n, gen, f, omega):
    make = synth.dominant_system if gen == "dom" else synth.hard_system
    A, B, _ = make(n, f, seed=1300 + n)
    s = solver(jac, A, B, omega=omega)
    for k in (1, 2, 5):
        X, st = s.solve(max_iter=k, tol=1e-300)
        ref = oracle.block_sor(A, B, max_iter=k, tol=1e-300, blocks=1, omega=omega)
        assert st.sweeps == ref.iters <= k  # a component change of exactly 0 stops early (n = 1)
        assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-12, k
    X, st = s.solve(max_iter=3000, tol=1e-12)
    ref = oracle.block_sor(A, B, max_iter=3000, tol=1e-12, blocks=1, omega=omega)
    assert (st.status, st.sweeps) == (ref.status, ref.iters)
    assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-12


def test_sor_result_does_not_depend_on_the_grid(jac):
    A, B, _ = synth.hard_system(1500, 1.05, seed=77)
    ref = oracle.block_sor(A, B, max_iter=3000, tol=1e-12, blocks=1)
    for grid in (14, 23, 64, 0):
        X, st = solver(jac, A, B, grid=grid).solve(max_iter=3000, tol=1e-12)
        assert st.sweeps == ref.iters, grid
        assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-12, grid


def test_sor_euclidean_norm(jac):
    A, B, _ = synth.dominant_system(500, 1.1, seed=78)
    X, st = solver(jac, A, B, norm="2").solve(max_iter=500, tol=1e-11)
    ref = oracle.block_sor(A, B, max_iter=500, tol=1e-11, norm=oracle.NORM_2, blocks=1)
    assert (st.status, st.sweeps) == (ref.status, ref.iters)
    assert abs(st.final_delta - ref.delta) <= 1e-9 * ref.delta + 1e-15


def test_sor_errors(jac):
    import torch
    A, B, _ = synth.dominant_system(64, 1.2, seed=79)
    with pytest.raises(jac.JacobiError) as e:
        jac.DeviceSolver(torch.from_numpy(A).cuda(), torch.from_numpy(B[:, 0].copy()).cuda(), precision="bf16_ir",
                         method="sor")
    assert e.value.status == jac.ERR_UNSUPPORTED
    with pytest.raises(jac.JacobiError) as e:
        solver(jac, A, B, omega=2.0)
    assert e.value.status == jac.ERR_INVALID_ARG
    A[5, 5] = 0.0
    with pytest.raises(jac.JacobiError) as e:
        solver(jac, A, B)
    assert e.value.status == jac.ERR_ZERO_DIAGONAL


def test_sor_full_size_hard_generator(jac):
    """n = 16384 on the paper-shaped generator (rho(T) = 1/1.05): Gauss-Seidel converges in a few dozen
    sweeps where Jacobi needs hundreds; 64 sampled rows of the residual are rechecked on the host."""
    n = 16384
    A, B, Xs = synth.hard_system(n, 1.05, seed=synth.BASE_SEED + 5)
    X, st = solver(jac, A, B).solve(max_iter=1000, tol=1e-13)
    assert st.status == 0 and st.sweeps < 40, st.as_dict()
    Xh = X.cpu().numpy()
    rows = np.random.default_rng(2).choice(n, size=64, replace=False)
    R = B[rows, 0] - A[rows] @ Xh
    assert np.max(np.abs(R)) / np.max(np.abs(B)) <= 1e-10
    assert np.max(np.abs(Xh - Xs[:, 0])) <= 1e-9


def test_sor_far_start_vector_takes_the_fp64_links(jac):
    """A start vector 1e40 times larger than max |b_i / a_ii| puts the first hand-offs outside the range of
    the float-float product (values at or above 2^(g + 100)), so those links run in FP64; the iterates still
    follow the oracle as the iteration contracts back to the solution's scale."""
    A, B, _ = synth.dominant_system(900, 1.1, seed=80)
    x0 = 1e40 * np.cos(np.arange(900.0))
    s = solver(jac, A, B)
    import torch
    for k in (1, 2, 5, 12):  # by sweep 12 the values are back inside the float-float range
        X, st = s.solve(X0=torch.from_numpy(x0).cuda(), max_iter=k, tol=1e-300)
        ref = oracle.block_sor(A, B, X0=x0[:, None], max_iter=k, tol=1e-300, blocks=1)
        assert st.sweeps == ref.iters == k
        assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-12, k


@pytest.mark.parametrize("case", range(8))
def test_sor_random_configurations(jac, case):
    """Seeded random mixes of size (ragged against the 112-row blocks), grid, omega, generator and norm:
    the iterate after 3 sweeps and the converged solve against the oracle."""
    rng = np.random.default_rng(900 + case)
    n = int(rng.integers(2, 2400))
    gen = synth.dominant_system if rng.random() < 0.6 else synth.hard_system
    f = float(rng.uniform(1.05, 1.5))
    omega = float(rng.choice([1.0, 1.0, float(rng.uniform(0.6, 1.4))]))
    norm = "2" if rng.random() < 0.3 else "inf"
    need = -(-n // 112)
    grid = int(rng.integers(need, max(need, min(152, n)) + 1)) if rng.random() < 0.5 else 0
    A, B, _ = gen(n, f, seed=1000 + case)
    s = solver(jac, A, B, omega=omega, norm=norm, grid=grid)
    onorm = oracle.NORM_2 if norm == "2" else oracle.NORM_INF
    X, st = s.solve(max_iter=3, tol=1e-300)
    ref = oracle.block_sor(A, B, max_iter=3, tol=1e-300, blocks=1, omega=omega, norm=onorm)
    assert st.sweeps == ref.iters
    assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-12, (n, grid, omega)
    X, st = s.solve(max_iter=3000, tol=1e-11)
    ref = oracle.block_sor(A, B, max_iter=3000, tol=1e-11, blocks=1, omega=omega, norm=onorm)
    assert st.status == ref.status == 0, (n, grid, omega, st.as_dict())
    assert abs(st.sweeps - ref.iters) <= (1 if norm == "2" else 0), (st.sweeps, ref.iters)
    assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-11


def test_sor_bounded_waits_expire_and_context_stays_usable(jac):
    """Failure detection without a GPU fault: block 0 never publishes its first sweep and raises the error
    word; the blocks waiting on its flag leave at once, the one polling its mailbox after its bounded wait
    (50 ms), the solve reports a timeout, and the next solve on the same context matches the oracle."""
    A, B, _ = synth.dominant_system(2000, 1.2, seed=81)
    flags = jac.binding.FLAG_SHORT_WAITS | jac.binding.FLAG_TEST_SKIP_ARRIVAL
    bad = solver(jac, A, B, flags=flags)
    with pytest.raises(jac.JacobiError) as e:
        bad.solve(max_iter=100, tol=1e-12)
    assert e.value.status == jac.ERR_TIMEOUT
    X, st = solver(jac, A, B).solve(max_iter=1000, tol=1e-12)
    ref = oracle.block_sor(A, B, max_iter=1000, tol=1e-12, blocks=1)
    assert (st.status, st.sweeps) == (ref.status, ref.iters)
    assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-12
