"""Many right-hand sides: the FP64 path (dense FP64 passes) and BF16 inner sweeps on tcgen05.

* FP64, r columns: every iterate within 1e-12 of the oracle's (which runs all columns together, max-norm
  over every entry), equal sweep count.
* The tcgen05 product itself: with one outer step and one inner sweep, X = c1 - f * (Q . bf16(c1)), where
  Q holds the oracle's BF16 codes of the off-diagonal part of A and f = fp32(1 / a_ii); the kernel
  accumulates in FP32, so the tolerance is FP32 rounding over n terms.
* BF16 refinement: ||B - A X||_inf / ||B||_inf <= 1e-10 for every column (oracle, FP64), and the error
  against the planted solution within the residual bound.
"""
import os

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


def dev(A, B):
    import torch
    return torch.from_numpy(A).cuda(), torch.from_numpy(np.ascontiguousarray(B.T)).cuda()


def bf16_values(codes):
    return (codes.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("n,r", [(100, 3), (300, 16), (517, 64)])
def test_fp64_many_rhs_matches_oracle(jac, n, r):
    A, B, _ = synth.dominant_system(n, 1.2, seed=600 + n, nrhs=r)
    At, Bt = dev(A, B)
    s = jac.MultiSolver(At, Bt, precision="fp64")
    for k in (1, 4):
        X, st = s.solve(max_iter=k, tol=1e-300)
        ref = oracle.jacobi(A, B, max_iter=k, tol=1e-300)
        assert st.sweeps == k
        err = np.max(np.abs(X.cpu().numpy().T - ref.X)) / np.max(np.abs(ref.X))
        assert err <= 1e-12, (k, err)
    X, st = s.solve(max_iter=1000, tol=1e-12)
    ref = oracle.jacobi(A, B, max_iter=1000, tol=1e-12)
    assert (st.status, st.sweeps) == (ref.status, ref.iters)
    assert np.max(np.abs(X.cpu().numpy().T - ref.X)) <= 1e-12 * np.max(np.abs(ref.X))


@pytest.mark.parametrize("n,r", [(256, 16), (300, 64), (1000, 32), (1536, 128), (20480, 64)])
def test_tcgen05_sweep_product(jac, n, r):
    # n = 20480: 160 row tiles on 152 SMs, so two tiles share an SM as at n = 32768
    A, B, _ = synth.dominant_system(n, 1.1, seed=700 + n, nrhs=r)
    At, Bt = dev(A, B)
    s = jac.MultiSolver(At, Bt, precision="bf16_ir", max_outer=2, max_inner=1)
    X, st = s.solve(max_iter=10, tol=1e-300)
    assert st.outer_steps == 2 and st.sweeps == 1
    got = X.cpu().numpy().T  # (n, r)
    d = np.diag(A)
    rinv = 1.0 / d
    c1 = (B * rinv[:, None]).astype(np.float32).astype(np.float64)
    c1h = bf16_values(np.array([[oracle.bf16_from_f32(v) for v in col] for col in c1.T.astype(np.float32)],
                               dtype=np.uint16)).T
    Q = bf16_values(oracle.offdiag_bf16(A))
    f = rinv.astype(np.float32).astype(np.float64)
    prod = Q @ c1h
    want = c1 - f[:, None] * prod
    scale = np.abs(f)[:, None] * (np.abs(Q) @ np.abs(c1h))  # size of the FP32-accumulated sum
    assert np.all(np.abs(got - want) <= 2e-6 * scale + 1e-12), np.max(np.abs(got - want) / (scale + 1e-300))


@pytest.mark.parametrize("tc", [False, True], ids=["fp64_resid", "tc_resid"])
@pytest.mark.parametrize("n,r,gen", [(300, 16, "dom"), (777, 64, "dom"), (1024, 64, "hard"), (2000, 32, "dom"),
                                     (333, 128, "dom")])
def test_bf16_refinement_many_rhs(jac, n, r, gen, tc):
    make = synth.dominant_system if gen == "dom" else synth.hard_system
    A, B, Xs = make(n, 1.1, seed=800 + n, nrhs=r)
    At, Bt = dev(A, B)
    s = jac.MultiSolver(At, Bt, precision="bf16_ir", tc_residual=tc)
    X, st = s.solve(max_iter=5000, tol=1e-10)
    Xh = X.cpu().numpy().T
    _, rel = oracle.residual(A, B, Xh)
    assert st.status == 0 and rel <= 1e-10, (st.as_dict(), rel)
    q = 1 / 1.1
    err = np.max(np.abs(Xh - Xs), axis=0)
    assert np.all(err <= 2e-10 * (1 + q) / (1 - q) * np.max(np.abs(Xs))), err.max()


@pytest.fixture(scope="module")
def full_size_system():
    """n = 32768, 64 right-hand sides, f = 1.1, and the oracle's FP64 Jacobi solution (all host cores,
    residual-norm stop 1e-12)."""
    n, r = 32768, 64
    A, B, Xs = synth.dominant_system(n, 1.1, seed=synth.BASE_SEED + 3, nrhs=r)
    ref = oracle.jacobi(A, B, max_iter=200, tol=1e-12, norm=oracle.NORM_RESID, nthreads=oracle.num_threads())
    assert ref.status == oracle.OK
    d = np.abs(np.diag(A))
    margin = float(np.min(d - (np.abs(A).sum(axis=1) - d)))
    return A, B, Xs, ref, margin


@pytest.mark.parametrize("tc", [False, True], ids=["fp64_resid", "tc_resid"])
def test_full_size_many_rhs_against_the_oracle(jac, full_size_system, tc):
    """n = 32768, 64 right-hand sides, f = 1.1 (the many-right-hand-side configuration at full size): BF16
    tcgen05 sweeps with FP64 refinement (the residual by FP64 FMAs, or on the tensor cores from the digit
    split), compared column by column with the oracle's FP64 Jacobi solve of the same system.  For strictly
    dominant A, ||A^-1||_inf <= 1 / min_i (|a_ii| - sum_{j!=i} |a_ij|), so two solutions whose residuals are
    at most 1e-10 and 1e-12 of ||b_c|| differ by at most ||A^-1||_inf (1e-10 + 1e-12) ||b_c||_inf in every
    entry (the oracle stops on its previous iterate's residual; the returned one is closer, as
    ||T||_inf < 1); a wrong entry anywhere in X fails that.  The residual of every column is also recomputed
    by the oracle on 512 sampled rows."""
    A, B, Xs, ref, margin = full_size_system
    n = A.shape[0]
    At, Bt = dev(A, B)
    s = jac.MultiSolver(At, Bt, precision="bf16_ir", tc_residual=tc)
    X, st = s.solve(max_iter=5000, tol=1e-10)
    assert st.status == 0 and st.rel_residual <= 1e-10
    Xh = X.cpu().numpy().T
    s.close()
    del At, Bt
    rows = np.random.default_rng(1).choice(n, size=512, replace=False)
    R = oracle.residual_rows(A, B, Xh, rows)
    bnorm = np.max(np.abs(B), axis=0)
    assert np.all(np.max(np.abs(R), axis=0) <= 1e-10 * bnorm), (np.max(np.abs(R), axis=0) / bnorm).max()
    # (+1e-12 for the rounding of the two FP64 residual evaluations, each ~sqrt(n) eps of ||b_c||)
    bound = (1e-10 + 2e-12) * bnorm / margin                      # per column
    err = np.max(np.abs(Xh - ref.X), axis=0)
    assert np.all(err <= bound), (err / bound).max()
    assert np.max(np.abs(ref.X - Xs)) <= 1e-12 * np.max(bnorm) / margin + 1e-13


def _one_residual(jac, A, B, X0, tc):
    """The per-column relative residuals ||b_c - A x0_c||_inf / ||b_c||_inf of one residual evaluation
    (max_outer = 1: the solve stops after it)."""
    import torch
    At, Bt = dev(A, B)
    s = jac.MultiSolver(At, Bt, precision="bf16_ir", tc_residual=tc, split_residual=not tc, max_outer=1)
    X0t = torch.from_numpy(np.ascontiguousarray(X0.T)).cuda()
    _, st = s.solve(X0=X0t, max_iter=10, tol=1e-300)
    assert st.outer_steps == 1 and st.sweeps == 0
    _, vals = s.column_stats()
    return np.asarray(vals)


@pytest.mark.parametrize("n,r", [(600, 16), (1000, 32), (517, 64), (300, 128), (2100, 16), (2500, 64)])
def test_tc_residual_wild_scales(jac, n, r):
    """The tensor-core residual (digit split of A and X) of a given X0, rows of A scaled by 2^-300 .. 2^300
    and columns of B (so of X) by 2^-200 .. 2^200, against the oracle's FP64 residual per column, within
    2^-44 of max_i sum_j |a_ij x_jc| / ||b_c|| (the split's bound is about 2^-50 of it; the rest is the
    oracle's own FP64 rounding).  n > 2048: three 1024-column chunks of K on a few row tiles, so each tile's
    K range is split over several CTAs and a second launch adds the parts."""
    A, B, Xs = synth.dominant_system(n, 1.3, seed=97 + n, nrhs=r)
    rng = np.random.default_rng(n)
    rows = 2.0 ** rng.integers(-300, 300, n)
    cols = 2.0 ** rng.integers(-200, 200, r)
    A = A * rows[:, None]
    B = B * rows[:, None] * cols[None, :]
    X0 = Xs * cols[None, :] * (1 + 1e-6 * rng.standard_normal((n, r)))
    got = _one_residual(jac, A, B, X0, tc=True)
    for c in range(r):
        _, rel = oracle.residual(A, B[:, c], X0[:, c])
        S = np.max(np.abs(A) @ np.abs(X0[:, c])) / np.max(np.abs(B[:, c]))
        assert rel > 1e-9 and abs(got[c] - rel) <= 2.0 ** -44 * S, (c, got[c], rel, S)


@pytest.mark.parametrize("n,r", [(512, 32), (2100, 16)])
def test_tc_residual_against_a_near_exact_residual(jac, n, r):
    """Where long double is IEEE quad precision (113-bit significand, as on Arm Linux), the residual of a
    hard-generator system (all entries of A positive: no cancellation in A x) is formed with exact products
    and 113-bit sums; the tensor-core residual must be within 2^-50 of max_i sum_j |a_ij x_jc| of it per
    column.  The BF16 digits are balanced, so a dropped digit or a wrong digit weight shows up far above
    that bound.  n = 2100: the K-split tiles (three chunks, partial sums added by a second launch)."""
    if np.finfo(np.longdouble).nmant < 105:
        pytest.skip("long double is not quad precision on this host")
    A, B, Xs = synth.hard_system(n, 1.2, seed=55, nrhs=r)
    X0 = Xs * (1 + 1e-7 * np.random.default_rng(3).standard_normal((n, r)))
    got = _one_residual(jac, A, B, X0, tc=True)
    Al, Bl, Xl = A.astype(np.longdouble), B.astype(np.longdouble), X0.astype(np.longdouble)
    R = Bl - Al @ Xl
    for c in range(r):
        want = float(np.max(np.abs(R[:, c])) / np.max(np.abs(Bl[:, c])))
        S = float(np.max(np.abs(Al) @ np.abs(Xl[:, c])) / np.max(np.abs(Bl[:, c])))
        assert abs(got[c] - want) <= 2.0 ** -50 * S, (c, got[c], want, S)


def test_fp64_many_rhs_residual_stop(jac):
    A, B, _ = synth.hard_system(400, 1.2, seed=611, nrhs=5)
    At, Bt = dev(A, B)
    s = jac.MultiSolver(At, Bt, precision="fp64", norm="resid")
    X, st = s.solve(max_iter=2000, tol=1e-10)
    ref = oracle.jacobi(A, B, max_iter=2000, tol=1e-10, norm=oracle.NORM_RESID)
    assert (st.status, st.sweeps) == (ref.status, ref.iters)
    assert np.max(np.abs(X.cpu().numpy().T - ref.X)) <= 1e-12 * np.max(np.abs(ref.X))


@pytest.mark.parametrize("n,r,gen", [(300, 16, "dom"), (777, 64, "dom"), (1024, 32, "hard"), (1536, 128, "dom")])
def test_split_residual_many_rhs(jac, n, r, gen):
    """BF16 refinement with the split-float residual (FP32 units): every column meets 1e-10 by the
    oracle's FP64 residual, and the reported residual matches it within the split's accuracy."""
    make = synth.dominant_system if gen == "dom" else synth.hard_system
    A, B, _ = make(n, 1.1, seed=900 + n, nrhs=r)
    At, Bt = dev(A, B)
    s = jac.MultiSolver(At, Bt, precision="bf16_ir", split_residual=True)
    X, st = s.solve(max_iter=5000, tol=1e-10)
    _, rel = oracle.residual(A, B, X.cpu().numpy().T)
    assert st.status == 0 and rel <= 1e-10, (st.as_dict(), rel)
    assert abs(st.rel_residual - rel) <= 5e-13 + 1e-3 * rel


def test_split_residual_many_rhs_wild_scales(jac):
    """One residual evaluation of a given X0 (max_outer = 1): rows of A scaled by 2^-300 .. 2^300 and
    columns of B (so of X) by 2^-200 .. 2^200; the split-float residual equals the oracle's FP64 one
    within the split's error bound."""
    import torch
    n, r = 600, 16
    A, B, Xs = synth.dominant_system(n, 1.3, seed=93, nrhs=r)
    rng = np.random.default_rng(5)
    rows = 2.0 ** rng.integers(-300, 300, n)
    cols = 2.0 ** rng.integers(-200, 200, r)
    A = A * rows[:, None]
    B = B * rows[:, None] * cols[None, :]
    X0 = Xs * cols[None, :] * (1 + 1e-6 * rng.standard_normal((n, r)))
    At, Bt = dev(A, B)
    s = jac.MultiSolver(At, Bt, precision="bf16_ir", split_residual=True, max_outer=1)
    X0t = torch.from_numpy(np.ascontiguousarray(X0.T)).cuda()
    _, st = s.solve(X0=X0t, max_iter=10, tol=1e-300)
    assert st.outer_steps == 1 and st.sweeps == 0
    _, rel = oracle.residual(A, B, X0)
    # the split's error bound: ~2^-46 of sum_j |a_ij x_jc| per row, relative to ||b_c||
    S = np.max((np.abs(A) @ np.abs(X0)).max(axis=0) / np.abs(B).max(axis=0))
    assert rel > 1e-9 and abs(st.rel_residual - rel) <= 2.0 ** -44 * S, (st.rel_residual, rel, S)


def test_fp64_column_retirement_matches_single_column_solves(jac):
    """Retiring columns: each column is the single-right-hand-side oracle solve of that column (same
    sweep count, iterate within 1e-12), whatever the other columns need."""
    n, r = 300, 6
    A, B, _ = synth.dominant_system(n, 1.2, seed=620, nrhs=r)
    B[:, 1] = 0.0      # X = 0 is exact: done after the first sweep
    B[:, 2] *= 1e-6    # the absolute change test is met sooner
    B[:, 4] *= 1e3     # and later
    At, Bt = dev(A, B)
    s = jac.MultiSolver(At, Bt, precision="fp64", retire_columns=True)
    X, st = s.solve(max_iter=1000, tol=1e-12)
    iters, vals = s.column_stats()
    Xh = X.cpu().numpy().T
    for c in range(r):
        ref = oracle.jacobi(A, B[:, c], max_iter=1000, tol=1e-12)
        assert ref.status == 0 and iters[c] == ref.iters, (c, iters[c], ref.iters)
        assert np.max(np.abs(Xh[:, c] - ref.X[:, 0])) <= 1e-12 * max(np.max(np.abs(ref.X)), 1e-300), c
    assert st.status == 0 and st.sweeps == iters.max()
    assert iters[1] == 1 and iters[2] < iters[0] < iters[4]


@pytest.mark.parametrize("tc,n", [(False, 777), (True, 777), (True, 2100)], ids=["fp64_resid", "tc_resid", "tc_resid_ksplit"])
def test_bf16_column_retirement(jac, tc, n):
    """Columns whose start vector already meets the target retire at the first residual evaluation and
    keep X0 bit for bit; the others refine on; every column ends at or below the 1e-10 target.  n = 2100
    with the tensor-core residual: its K-split tiles, whose second launch takes only the active columns."""
    import torch
    r = 16
    A, B, Xs = synth.dominant_system(n, 1.1, seed=621, nrhs=r)
    X0 = np.zeros((n, r))
    X0[:, ::2] = Xs[:, ::2]
    At, Bt = dev(A, B)
    X0t = torch.from_numpy(np.ascontiguousarray(X0.T)).cuda()
    s = jac.MultiSolver(At, Bt, precision="bf16_ir", retire_columns=True, tc_residual=tc)
    X, st = s.solve(X0=X0t, max_iter=5000, tol=1e-10)
    iters, vals = s.column_stats()
    Xh = X.cpu().numpy().T
    assert st.status == 0
    assert np.all(iters[::2] == 1) and np.all(iters[1::2] > 1)
    np.testing.assert_array_equal(Xh[:, ::2], X0[:, ::2])
    for c in range(r):
        _, rel = oracle.residual(A, B[:, c], Xh[:, c])
        assert rel <= 1e-10, (c, rel)
        assert abs(vals[c] - rel) <= 1e-13 + 1e-3 * rel


def test_fp64_many_rhs_euclidean_norm(jac):
    """Section 2's Euclidean stopping test on many right-hand sides: per column the square root of the
    summed squared changes, the stop on the largest column (as the oracle); with retirement, each column
    is the single-column oracle solve under the same norm.  Per-column values agree with the oracle's
    within the few-ulp rounding differences of the iterates (times sqrt(n))."""
    n, r = 500, 7
    A, B, _ = synth.dominant_system(n, 1.15, seed=630, nrhs=r)
    B[:, 3] *= 1e-4
    At, Bt = dev(A, B)
    s = jac.MultiSolver(At, Bt, precision="fp64", norm="2")
    X, st = s.solve(max_iter=2000, tol=1e-11)
    ref = oracle.jacobi(A, B, max_iter=2000, tol=1e-11, norm=oracle.NORM_2)
    assert (st.status, st.sweeps) == (ref.status, ref.iters)
    assert np.max(np.abs(X.cpu().numpy().T - ref.X)) <= 1e-12 * np.max(np.abs(ref.X))
    assert abs(st.final_delta - ref.delta) <= 2 * np.sqrt(n) * 1e-14
    s = jac.MultiSolver(At, Bt, precision="fp64", norm="2", retire_columns=True)
    X, st = s.solve(max_iter=2000, tol=1e-11)
    iters, vals = s.column_stats()
    Xh = X.cpu().numpy().T
    for c in range(r):
        ref = oracle.jacobi(A, B[:, c], max_iter=2000, tol=1e-11, norm=oracle.NORM_2)
        assert ref.status == 0 and iters[c] == ref.iters, (c, iters[c], ref.iters)
        assert np.max(np.abs(Xh[:, c] - ref.X[:, 0])) <= 1e-12 * np.max(np.abs(ref.X)), c
    assert iters[3] < iters[0]
