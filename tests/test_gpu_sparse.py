"""Sparse (CSR) Jacobi on the GPU against the CPU oracle's csr_jacobi.

The GPU keeps A as a sliced-ELL copy of its off-diagonal part and multiplies by 1 / a_ii; the oracle
divides and sums the stored entries in the same ascending column order.  Iterates must agree within
1e-12 (relative max-norm) after 1, 2 and 5 sweeps, with the same sweep count to convergence, on
irregular rows (empty, short and long) and on 1-D / 2-D / 3-D stencils whose size leaves a ragged last
slice.  The full-size 2-D workload is checked sweep by sweep for three sweeps, and its converged result
on sampled rows.
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


def gpu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_err(x, ref):
    return np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300)


SYSTEMS = {
    "irregular_1000": lambda: synth.random_sparse_system(1000, 1.1, seed=31, max_len=60),
    "irregular_33": lambda: synth.random_sparse_system(33, 1.3, seed=32, max_len=40),
    "long_rows_2000": lambda: synth.random_sparse_system(2000, 1.05, seed=39, max_len=1500),
    "one_unknown": lambda: synth.random_sparse_system(1, 1.5, seed=33),
    "line_95": lambda: synth.stencil_system((95,), 1.05, seed=34),
    "plane_37x29": lambda: synth.stencil_system((37, 29), 1.05, seed=35),
    "box_11x9x7": lambda: synth.stencil_system((11, 9, 7), 1.1, seed=36),
}


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_sparse_iterates_match_the_oracle(jac, name):
    rp, ci, v, B, _ = SYSTEMS[name]()
    s = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]))
    for k in (1, 2, 5):
        X, st = s.solve(max_iter=k, tol=1e-300)
        ref = oracle.csr_jacobi(rp, ci, v, B, max_iter=k, tol=1e-300)
        assert st.sweeps == ref.iters <= k
        assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-12, k
    X, st = s.solve(max_iter=5000, tol=1e-12)
    ref = oracle.csr_jacobi(rp, ci, v, B, max_iter=5000, tol=1e-12)
    assert (st.status, st.sweeps) == (ref.status, ref.iters)
    assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-12


def test_sparse_euclidean_norm_and_start_vector(jac):
    rp, ci, v, B, Xs = synth.stencil_system((40, 33), 1.2, seed=37)
    x0 = Xs[:, 0] + 1e-3 * np.sin(np.arange(B.shape[0]))
    s = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]), norm="2")
    X, st = s.solve(X0=gpu(x0), max_iter=2000, tol=1e-11)
    ref = oracle.csr_jacobi(rp, ci, v, B, X0=x0, max_iter=2000, tol=1e-11, norm=oracle.NORM_2)
    assert (st.status, st.sweeps) == (ref.status, ref.iters)
    # delta is the norm of a difference of nearly equal iterates, so it inherits their rounding
    # differences: the GPU sweep x = c + T x (rounded t_ij and c_i) and the oracle's (b - s) / a_ii differ by a
    # few ulps of max|x| per component and sweep, at most (w + 2) ulp / (1 - rho) ~ 1e-14 here (w <= 4,
    # rho <= 1/1.2), and | ||e_k|| - ||e_k'|| | <= ||e_k - e_k'||_2 <= 2 sqrt(n) max_i |x_i - x_i'|
    n = B.shape[0]
    assert abs(st.final_delta - ref.delta) <= 2 * np.sqrt(n) * 1e-14
    assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-12


def test_sparse_host_arrays_and_cap(jac):
    """numpy inputs (copied during setup), a host X_out, and the iteration cap: X^(L), NOT_CONVERGED."""
    import torch
    rp, ci, v, B, _ = synth.random_sparse_system(500, 1.02, seed=38, max_len=30)
    s = jac.CsrSolver(rp, ci, v, B[:, 0])
    out = torch.zeros(500, dtype=torch.float64)
    s.solve_async(max_iter=7, tol=1e-300, out=out)
    st = s.last_stats()
    ref = oracle.csr_jacobi(rp, ci, v, B, max_iter=7, tol=1e-300)
    assert st.status == ref.status == jac.NOT_CONVERGED and st.sweeps == 7
    assert rel_err(out.numpy(), ref.X[:, 0]) <= 1e-12


def test_sparse_errors_follow_the_oracle(jac):
    rp = np.array([0, 2, 4, 6], dtype=np.int64)
    ci = np.array([0, 1, 0, 1, 1, 2], dtype=np.int32)
    v = np.array([4.0, 1.0, 1.0, 4.0, 1.0, 4.0])
    b = np.ones(3)
    cases = []
    bad = ci.copy()
    bad[[4, 5]] = [2, 1]
    cases.append((rp, bad, v))                                   # descending columns
    bad = ci.copy()
    bad[5] = 3
    cases.append((rp, bad, v))                                   # column out of range
    cases.append((np.array([0, 4, 2, 6], dtype=np.int64), ci, v))  # decreasing row range
    z = v.copy()
    z[3] = 0.0
    cases.append((rp, ci, z))                                    # zero diagonal
    z = v.copy()
    z[3] = np.nan
    cases.append((rp, ci, z))                                    # non-finite diagonal
    cases.append((np.array([0, 2, 4, 5], dtype=np.int64), ci[:5].copy(), v[:5].copy()))  # missing diagonal
    for rp_, ci_, v_ in cases:
        want = oracle.csr_jacobi(rp_, ci_, v_, b).status
        with pytest.raises(jac.JacobiError) as e:
            jac.CsrSolver(rp_, ci_, v_, b)
        assert e.value.status == want, (rp_, ci_, v_)


def test_sparse_full_size_plane(jac):
    """The bench workload: 2-D variable-coefficient stencil on 2048 x 2048 (4.19 M unknowns), f = 1.05.
    Every iterate of the first three sweeps against the oracle; then the converged solve against the
    planted solution and the FP64 residual of 4096 sampled rows."""
    rp, ci, v, B, Xs = synth.stencil_system((2048, 2048), 1.05, seed=synth.BASE_SEED + 6)
    n = B.shape[0]
    s = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]))
    info = s.info()  # the 5-point stencil lies on 4 diagonals: stored diagonal by diagonal
    assert info["format"] == "dia" and info["diagonals"] == 4
    assert info["slices"] == n // 32 and info["stored_slots"] == 4 * n
    ell = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]), flags=jac.binding.FLAG_CSR_ELL).info()
    slot_width = (np.diff(rp) - 1).reshape(-1, 32).max(axis=1)  # each slice as wide as its longest row
    assert ell["format"] == "ell" and ell["stored_slots"] == 32 * int(slot_width.sum())
    X, st = s.solve(max_iter=3, tol=1e-300)
    ref = oracle.csr_jacobi(rp, ci, v, B, max_iter=3, tol=1e-300)
    assert st.sweeps == 3 and rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-12
    X, st = s.solve(max_iter=2000, tol=1e-12)
    assert st.status == 0 and 400 < st.sweeps < 700, st.as_dict()
    Xh = X.cpu().numpy()
    rows = np.random.default_rng(3).choice(n, size=4096, replace=False)
    r = np.array([B[i, 0] - v[rp[i]:rp[i + 1]] @ Xh[ci[rp[i]:rp[i + 1]]] for i in rows])
    assert np.max(np.abs(r)) / np.max(np.abs(B)) <= 1e-11
    assert np.max(np.abs(Xh - Xs[:, 0])) <= 1e-10


def test_sparse_bounded_wait_expires_and_context_stays_usable(jac):
    """Failure detection without a GPU fault: CTA 0 skips the first sweep's grid barrier and raises the
    error word, the other CTAs leave their bounded wait (50 ms at most), the solve reports a timeout, and
    the next solve on the same context matches the oracle."""
    rp, ci, v, B, _ = synth.stencil_system((300, 200), 1.1, seed=40)
    flags = jac.binding.FLAG_SHORT_WAITS | jac.binding.FLAG_TEST_SKIP_ARRIVAL
    bad = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]), flags=flags)
    assert bad.info()["grid"] > 1
    with pytest.raises(jac.JacobiError) as e:
        bad.solve(max_iter=100, tol=1e-12)
    assert e.value.status == jac.ERR_TIMEOUT
    good = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]))
    X, st = good.solve(max_iter=2000, tol=1e-12)
    ref = oracle.csr_jacobi(rp, ci, v, B, max_iter=2000, tol=1e-12)
    assert (st.status, st.sweeps) == (ref.status, ref.iters)
    assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-12


@pytest.mark.parametrize("case", range(8))
def test_sparse_random_configurations(jac, case):
    """Seeded random mixes of stencil shape / irregular rows, size, dominance, norm and start vector: the
    iterate after 3 sweeps and the converged solve against the oracle."""
    rng = np.random.default_rng(700 + case)
    kind = rng.integers(0, 4)
    f = float(rng.uniform(1.02, 1.5))
    if kind == 0:
        rp, ci, v, B, Xs = synth.random_sparse_system(int(rng.integers(1, 5000)), f, seed=800 + case,
                                                      max_len=int(rng.integers(1, 200)))
    else:
        shape = tuple(int(x) for x in rng.integers(1, [4000, 90, 22][kind - 1], size=kind))
        rp, ci, v, B, Xs = synth.stencil_system(shape, f, seed=800 + case)
    n = B.shape[0]
    norm = "2" if rng.random() < 0.3 else "inf"
    onorm = oracle.NORM_2 if norm == "2" else oracle.NORM_INF
    x0 = None if rng.random() < 0.5 else rng.uniform(-2, 2, n)
    s = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]), norm=norm)
    X, st = s.solve(X0=None if x0 is None else gpu(x0), max_iter=3, tol=1e-300)
    ref = oracle.csr_jacobi(rp, ci, v, B, X0=x0, max_iter=3, tol=1e-300, norm=onorm)
    assert st.sweeps == ref.iters
    assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-12, (n, kind)
    X, st = s.solve(X0=None if x0 is None else gpu(x0), max_iter=20000, tol=1e-11)
    ref = oracle.csr_jacobi(rp, ci, v, B, X0=x0, max_iter=20000, tol=1e-11, norm=onorm)
    assert st.status == ref.status == 0, (n, kind, st.as_dict())
    assert abs(st.sweeps - ref.iters) <= (1 if norm == "2" else 0), (st.sweeps, ref.iters)
    assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-11


# ---- mixed precision: FP32 / BF16 inner sweeps, FP64 refinement -----------------------------------------

@pytest.mark.parametrize("prec", ["fp32_ir", "bf16_ir"])
@pytest.mark.parametrize("name", ["irregular_1000", "irregular_33", "one_unknown", "line_95", "plane_37x29",
                                  "box_11x9x7", "long_rows_2000"])
def test_sparse_ir_meets_the_residual_target(jac, prec, name):
    """Refined to ||b - A x||_inf / ||b||_inf <= 1e-10, recomputed by the CSR oracle in FP64, and the
    solve's own reported residual agrees with it."""
    rp, ci, v, B, Xs = SYSTEMS[name]()
    s = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]), precision=prec)
    X, st = s.solve(max_iter=1, tol=1e-10)
    _, rel = oracle.csr_residual(rp, ci, v, B, X.cpu().numpy())
    assert st.status == 0 and rel <= 1e-10, (st.as_dict(), rel)
    assert abs(st.rel_residual - rel) <= 1e-3 * 1e-10
    assert st.outer_steps >= 1 and st.sweeps >= st.outer_steps - 1


def test_sparse_ir_full_size_plane(jac):
    """The bench workload in BF16 inner precision: the FP64 residual of every row, checked by the oracle,
    and the error against the planted solution."""
    rp, ci, v, B, Xs = synth.stencil_system((2048, 2048), 1.05, seed=synth.BASE_SEED + 6)
    s = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]), precision="bf16_ir")
    X, st = s.solve(max_iter=1, tol=1e-10)
    Xh = X.cpu().numpy()
    _, rel = oracle.csr_residual(rp, ci, v, B, Xh)
    assert st.status == 0 and rel <= 1e-10, (st.as_dict(), rel)
    assert np.max(np.abs(Xh - Xs[:, 0])) <= 1e-8


def test_sparse_ir_cap_errors_and_timeout(jac):
    import torch
    rp, ci, v, B, _ = synth.stencil_system((60, 50), 1.05, seed=41)
    # the outer cap: X is the last refined iterate, NOT_CONVERGED
    s = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]), precision="bf16_ir", max_outer=1)
    out = torch.empty(B.shape[0], dtype=torch.float64, device="cuda")
    s.solve_async(max_iter=1, tol=1e-14, out=out)
    st = s.last_stats()
    _, rel = oracle.csr_residual(rp, ci, v, B, out.cpu().numpy())
    assert st.status == jac.NOT_CONVERGED and st.outer_steps == 2 and abs(st.rel_residual - rel) <= 1e-6 * rel
    with pytest.raises(jac.JacobiError) as e:
        jac.CsrSolver(rp, ci, v, B[:, 0], precision="fp8_ir")
    assert e.value.status == jac.ERR_UNSUPPORTED
    with pytest.raises(jac.JacobiError) as e:
        jac.CsrSolver(rp, ci, v, B[:, 0], precision="fp32_ir", norm="2")
    assert e.value.status == jac.ERR_INVALID_ARG
    flags = jac.binding.FLAG_SHORT_WAITS | jac.binding.FLAG_TEST_SKIP_ARRIVAL
    bad = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]), precision="fp32_ir", flags=flags)
    with pytest.raises(jac.JacobiError) as e:
        bad.solve(max_iter=1, tol=1e-10)
    assert e.value.status == jac.ERR_TIMEOUT
    X, st = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]), precision="fp32_ir").solve(max_iter=1, tol=1e-10)
    assert st.status == 0 and oracle.csr_residual(rp, ci, v, B, X.cpu().numpy())[1] <= 1e-10


def test_sparse_residual_norm_stop(jac):
    """JACOBI_NORM_RESID on the FP64 path: the stop on ||b - A x^(k-1)|| / ||b|| follows the oracle's sweep
    count; the reported value carries the iterates' few-ulp rounding differences (times a_ii / ||b||)."""
    rp, ci, v, B, _ = synth.random_sparse_system(1500, 1.05, seed=42, max_len=40)
    s = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]), norm="resid")
    X, st = s.solve(max_iter=5000, tol=1e-10)
    ref = oracle.csr_jacobi(rp, ci, v, B, max_iter=5000, tol=1e-10, norm=oracle.NORM_RESID)
    assert (st.status, st.sweeps) == (ref.status, ref.iters)
    assert abs(st.final_delta - ref.delta) <= 1e-3 * ref.delta
    assert rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-12
    _, rel = oracle.csr_residual(rp, ci, v, B, X.cpu().numpy())
    assert rel < 1e-10


def test_sparse_divergence_follows_the_oracle(jac):
    """f = 0.9: rho(T) > 1.  At a cap of 200 sweeps both return X^(200) with JACOBI_NOT_CONVERGED; without
    a cap the iterates overflow and both stop with JACOBI_ERR_NONFINITE, within the few sweeps by which
    the two forms of the row sum move the overflow."""
    rp, ci, v, B, _ = synth.stencil_system((40, 30), 0.9, seed=44)
    s = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]))
    import torch
    out = torch.empty(B.shape[0], dtype=torch.float64, device="cuda")
    s.solve_async(max_iter=200, tol=1e-12, out=out)
    st = s.last_stats()
    ref = oracle.csr_jacobi(rp, ci, v, B, max_iter=200, tol=1e-12)
    assert (st.status, st.sweeps) == (ref.status, ref.iters) == (jac.NOT_CONVERGED, 200)
    assert rel_err(out.cpu().numpy(), ref.X[:, 0]) <= 1e-12
    ref200 = ref.X[:, 0]
    s.solve_async(max_iter=20000, tol=1e-12, out=out)
    st = s.last_stats()
    ref = oracle.csr_jacobi(rp, ci, v, B, max_iter=20000, tol=1e-12)
    assert st.status == ref.status == jac.ERR_NONFINITE
    # The sweep at which the iterate overflows depends on the form of the row sum.  The oracle forms
    # sum_j a_ij x_j, up to max_i sum_j |a_ij| times ||x||_inf, before dividing by a_ii; the GPU adds
    # t_ij x_j terms that are already divided.  The two overflow points differ by at most a factor of
    # that row sum (times |a_ii|, which is at least 1 here) in ||x||, i.e. by log(row sum) / log(growth)
    # sweeps at the growth per sweep seen in the oracle, plus one sweep either side for rounding.
    A = synth.csr_to_dense(B.shape[0], rp, ci, v)
    nxt = oracle.csr_jacobi(rp, ci, v, B, max_iter=201, tol=1e-300).X[:, 0]
    growth = np.max(np.abs(nxt)) / np.max(np.abs(ref200))
    window = np.log(np.abs(A).sum(axis=1).max()) / np.log(growth) + 2
    assert abs(st.sweeps - ref.iters) <= window, (st.sweeps, ref.iters, window)


# ---- storage formats: DIA for entries on a few diagonals, sliced ELL otherwise ----------------------------

def banded_system(n, offsets, f, seed):
    """Off-diagonals uniform [-1, 1) on the given diagonals (where they fall inside the matrix), a_ii = f *
    row sum of |a_ij|, planted X* and B = A X*, as CSR."""
    rng = np.random.default_rng(seed)
    A = np.zeros((n, n))
    for off in offsets:
        i = np.arange(max(0, -off), min(n, n - off))
        A[i, i + off] = rng.uniform(-1, 1, i.size)
    A[np.arange(n), np.arange(n)] = f * np.abs(A).sum(axis=1) + (np.abs(A).sum(axis=1) == 0)
    return dense_to_csr(A) + (A,)


def dense_to_csr(A):
    r, c = np.nonzero(A)
    rp = np.zeros(A.shape[0] + 1, dtype=np.int64)
    np.add.at(rp, r + 1, 1)
    rp = np.cumsum(rp)
    Xs = np.random.default_rng(5).uniform(-1, 1, (A.shape[0], 1))
    return rp, c.astype(np.int32), A[r, c].copy(), A @ Xs


@pytest.mark.parametrize("prec", ["fp64", "bf16_ir", "fp32_ir"])
@pytest.mark.parametrize("name,ndiag", [("line_95", 2), ("plane_37x29", 4), ("box_11x9x7", 6)])
def test_dia_and_ell_give_the_same_solves(jac, prec, name, ndiag):
    """A stencil is kept in DIA form (no column array, contiguous gathers) unless sliced ELL is asked for.
    The two sum the same entries in the same column order (DIA's absent entries are zeros), so every
    iterate and the converged result are equal, and both follow the oracle."""
    rp, ci, v, B, _ = SYSTEMS[name]()
    dia = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]), precision=prec)
    ell = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]), precision=prec, flags=jac.binding.FLAG_CSR_ELL)
    assert (dia.info()["format"], dia.info()["diagonals"]) == ("dia", ndiag)
    assert (ell.info()["format"], ell.info()["diagonals"]) == ("ell", 0)
    caps = (1, 3, 5000) if prec == "fp64" else (5000,)
    tol = 1e-12 if prec == "fp64" else 1e-10
    for cap in caps:
        Xd, sd = dia.solve(max_iter=cap, tol=tol if cap > 10 else 1e-300)
        Xe, se = ell.solve(max_iter=cap, tol=tol if cap > 10 else 1e-300)
        assert (sd.status, sd.sweeps, sd.outer_steps) == (se.status, se.sweeps, se.outer_steps)
        np.testing.assert_array_equal(Xd.cpu().numpy(), Xe.cpu().numpy())
    if prec == "fp64":
        ref = oracle.csr_jacobi(rp, ci, v, B, max_iter=5000, tol=1e-12)
        assert sd.sweeps == ref.iters and rel_err(Xd.cpu().numpy(), ref.X[:, 0]) <= 1e-12
    else:
        assert sd.status == 0 and oracle.csr_residual(rp, ci, v, B, Xd.cpu().numpy())[1] <= 1e-10


@pytest.mark.parametrize("offsets,fmt", [((-1, 1), "dia"), ((-300, -7, -1, 1, 2, 40, 299), "dia"),
                                         (tuple(range(-8, 0)) + tuple(range(1, 9)), "dia"),
                                         (tuple(range(-9, 0)) + tuple(range(1, 9)), "ell")])
def test_banded_matrices_pick_dia_up_to_16_diagonals(jac, offsets, fmt):
    n = 1000
    rp, ci, v, B, A = banded_system(n, offsets, 1.1, seed=len(offsets))
    s = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]))
    assert s.info()["format"] == fmt
    for k in (1, 4):
        X, st = s.solve(max_iter=k, tol=1e-300)
        ref = oracle.csr_jacobi(rp, ci, v, B, max_iter=k, tol=1e-300)
        assert st.sweeps == ref.iters and rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-12
    X, st = s.solve(max_iter=5000, tol=1e-12)
    ref = oracle.csr_jacobi(rp, ci, v, B, max_iter=5000, tol=1e-12)
    assert (st.status, st.sweeps) == (ref.status, ref.iters) and rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-12


def test_an_entry_off_the_sampled_diagonals_keeps_ell(jac):
    """Setup takes candidate diagonals from a few rows and then checks every entry: one entry elsewhere
    (in a row it did not sample) keeps the matrix in sliced ELL, and the solve still follows the oracle."""
    rp0, ci0, v0, B0, _ = synth.stencil_system((40, 33), 1.2, seed=41)
    A = synth.csr_to_dense(B0.shape[0], rp0, ci0, v0)
    A[5, 900] = -0.01
    A[5, 5] += 0.02
    rp, ci, v, B = dense_to_csr(A)
    s = jac.CsrSolver(gpu(rp), gpu(ci), gpu(v), gpu(B[:, 0]))
    assert s.info()["format"] == "ell"
    X, st = s.solve(max_iter=5000, tol=1e-12)
    ref = oracle.csr_jacobi(rp, ci, v, B, max_iter=5000, tol=1e-12)
    assert (st.status, st.sweeps) == (ref.status, ref.iters) and rel_err(X.cpu().numpy(), ref.X[:, 0]) <= 1e-12
