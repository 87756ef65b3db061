"""Batched uneven systems (one system per CTA, work queue, graph replay) against the CPU oracle.

FP64 mode is the Section 2 iteration with the previous-iterate relative-residual stop: each system's
sweep count equals the oracle's and its X is within 1e-12 (relative max-norm) of the oracle's.
Mixed modes: each system's ||B - A X||_inf / ||B||_inf <= tol, recomputed by the oracle in FP64, and
its error against the oracle's converged FP64 solution within the residual bound.  Each system's result
is the same alone as in the mix.
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


def make_batch(count, n_lo, n_hi, f_lo, f_hi, seed, gen="dom"):
    ns, fs = synth.batch_shapes(count, n_lo, n_hi, f_lo, f_hi, seed)
    make = synth.dominant_system if gen == "dom" else synth.hard_system
    systems = [make(int(n), float(f), synth.system_seed(seed, k)) for k, (n, f) in enumerate(zip(ns, fs))]
    return systems


def to_dev(systems):
    import torch
    As = [torch.from_numpy(A).cuda() for A, _, _ in systems]
    Bs = [torch.from_numpy(B[:, 0].copy()).cuda() for _, B, _ in systems]
    return As, Bs


def qnorm(A):
    M = np.abs(A)
    d = np.diag(M).copy()
    np.fill_diagonal(M, 0.0)
    return float(np.max(M.sum(axis=1) / d))


@pytest.mark.parametrize("rpw", [1, 4, 8])
def test_fp64_batch_matches_oracle(jac, rpw):
    systems = make_batch(37, 1, 300, 1.05, 2.0, seed=101)
    systems.append(synth.hard_system(257, 1.1, seed=7))
    As, Bs = to_dev(systems)
    tol = 1e-10
    bs = jac.BatchSolver(As, Bs, precision="fp64", rows_per_warp=rpw)
    X = bs.solve_async(max_iter=3000, tol=tol)
    stats = bs.stats()
    for k, (A, B, _) in enumerate(systems):
        ref = oracle.jacobi(A, B, max_iter=3000, tol=tol, norm=oracle.NORM_RESID)
        st = stats[k]
        assert (st.status, st.sweeps) == (ref.status, ref.iters), (k, A.shape[0])
        x = X[k].cpu().numpy()
        assert np.max(np.abs(x - ref.X[:, 0])) <= 1e-12 * np.max(np.abs(ref.X)), k


@pytest.mark.parametrize("prec", ["fp64", "fp32_ir", "bf16_ir"])
def test_batch_rows_not_16_byte_aligned(jac, prec):
    """A given 8 bytes past a 16-byte boundary (a view one element into a larger buffer), with even and odd
    n: the kernel's 8-byte load paths.  FP64 against the oracle (sweep count, X within 1e-12); the mixed
    modes reach the target, rechecked by the oracle."""
    import torch
    systems = make_batch(12, 2, 400, 1.05, 2.0, seed=707)
    systems += [synth.dominant_system(n, 1.1, seed=708 + n) for n in (64, 256, 1000)]
    As, Bs = [], []
    for A, B, _ in systems:
        n = A.shape[0]
        buf = torch.zeros(n * n + 1, dtype=torch.float64, device="cuda")
        buf[1:] = torch.from_numpy(A.ravel()).cuda()
        As.append(buf[1:].view(n, n))
        Bs.append(torch.from_numpy(B[:, 0].copy()).cuda())
    assert all(a.data_ptr() % 16 == 8 for a in As)
    bs = jac.BatchSolver(As, Bs, precision=prec)
    X = bs.solve_async(max_iter=5000, tol=1e-10)
    stats = bs.stats()
    for k, (A, B, _) in enumerate(systems):
        x = X[k].cpu().numpy()
        if prec == "fp64":
            ref = oracle.jacobi(A, B, max_iter=5000, tol=1e-10, norm=oracle.NORM_RESID)
            assert (stats[k].status, stats[k].sweeps) == (ref.status, ref.iters), (k, A.shape[0])
            assert np.max(np.abs(x - ref.X[:, 0])) <= 1e-12 * np.max(np.abs(ref.X)), k
        else:
            _, rel = oracle.residual(A, B, x)
            assert stats[k].status == 0 and rel <= 1e-10, (k, A.shape[0], rel)


@pytest.mark.parametrize("prec,split", [("fp32_ir", False), ("bf16_ir", False), ("fp32_ir", True), ("bf16_ir", True)])
def test_mixed_batch_reaches_target(jac, prec, split):
    """split: residuals with the split-float arithmetic (FP32 units) instead of FP64 FMAs."""
    systems = make_batch(45, 1, 600, 1.05, 2.0, seed=202)
    systems.append(synth.hard_system(400, 1.1, seed=8))
    As, Bs = to_dev(systems)
    bs = jac.BatchSolver(As, Bs, precision=prec, split_residual=split)
    X = bs.solve_async(max_iter=5000, tol=1e-10)
    stats = bs.stats()
    for k, (A, B, _) in enumerate(systems):
        x = X[k].cpu().numpy()
        _, rel = oracle.residual(A, B, x)
        st = stats[k]
        assert st.status == 0 and rel <= 1e-10, (k, A.shape[0], st.as_dict(), rel)
        assert abs(st.rel_residual - rel) <= (5e-13 if split else 1e-13) + 1e-3 * rel
        q = qnorm(A)
        ref = oracle.jacobi(A, B, max_iter=20000, tol=1e-14)
        err = np.max(np.abs(x - ref.X[:, 0])) / np.max(np.abs(ref.X))
        assert err <= 2e-10 * (1 + q) / (1 - q) + 1e-13, (k, err)


@pytest.mark.parametrize("split", [False, True])
def test_alone_equals_in_the_mix_and_replay_is_bitwise(jac, split):
    import torch
    systems = make_batch(20, 50, 400, 1.05, 2.0, seed=303)
    As, Bs = to_dev(systems)
    mix = jac.BatchSolver(As, Bs, precision="fp32_ir", split_residual=split)
    X1 = [x.clone() for x in mix.solve_async(max_iter=5000, tol=1e-10)]
    X2 = [x.clone() for x in mix.solve_async(max_iter=5000, tol=1e-10)]
    for a, b in zip(X1, X2):
        assert torch.equal(a, b)
    for k in (0, 7, 19):
        alone = jac.BatchSolver([As[k]], [Bs[k]], precision="fp32_ir", split_residual=split)
        Xa = alone.solve_async(max_iter=5000, tol=1e-10)[0]
        # one CTA runs a system the same way whatever else is in the batch: identical bits
        assert torch.equal(Xa, X1[k])


def test_bad_system_does_not_disturb_the_others(jac):
    systems = make_batch(6, 10, 80, 1.2, 1.5, seed=404)
    A_bad = np.eye(5)
    A_bad[2, 2] = 0.0
    systems.insert(3, (A_bad, np.ones((5, 1)), None))
    As, Bs = to_dev(systems)
    bs = jac.BatchSolver(As, Bs, precision="fp32_ir")
    X = bs.solve_async(max_iter=1000, tol=1e-10)
    stats = bs.stats()
    assert stats[3].status == jac.ERR_ZERO_DIAGONAL
    for k, (A, B, _) in enumerate(systems):
        if k == 3:
            continue
        _, rel = oracle.residual(A, B, X[k].cpu().numpy())
        assert stats[k].status == 0 and rel <= 1e-10


@pytest.mark.parametrize("prec", ["fp32_ir", "fp64"])
def test_zero_right_hand_side_in_the_mix(jac, prec):
    """One system with B = 0 (solution X = 0) among ordinary ones.  Both batch modes stop on the relative
    residual ||B - A X|| / ||B||, which is 0 / 0 there: that system reports JACOBI_ERR_NONFINITE with X = 0,
    as the oracle's residual-norm stop does, and the others are not disturbed."""
    import torch
    systems = make_batch(6, 10, 80, 1.2, 1.5, seed=405)
    A0, _, _ = synth.dominant_system(50, 1.3, seed=406)
    systems.insert(2, (A0, np.zeros((50, 1)), None))
    As, Bs = to_dev(systems)
    bs = jac.BatchSolver(As, Bs, precision=prec)
    X = bs.solve_async(max_iter=1000, tol=1e-10)
    stats = bs.stats()
    ref = oracle.jacobi(A0, np.zeros(50), max_iter=1000, tol=1e-10, norm=oracle.NORM_RESID)
    assert stats[2].status == ref.status == jac.ERR_NONFINITE
    assert int(torch.count_nonzero(X[2])) == 0
    for k, (A, B, _) in enumerate(systems):
        if k == 2:
            continue
        _, rel = oracle.residual(A, B, X[k].cpu().numpy())
        assert stats[k].status == 0 and rel <= 1e-10


@pytest.mark.parametrize("prec,shape", [("fp32_ir", {}), ("fp32_ir", {"rows_per_warp": 4, "ctas_per_sm": 4,
                                                                    "inner_rtol": 2.0 ** -10}),
                                        ("fp64", {"rows_per_warp": 8, "ctas_per_sm": 4})],
                         ids=["fp32_ir_defaults", "fp32_ir_bench_shape", "fp64_bench_shape"])
def test_full_size_batch_sampled(jac, prec, shape):
    """4096 systems, n log-uniform in [64, 1024], f uniform in [1.05, 2.0]: FP32 storage with FP64 refinement
    (the descriptor defaults, and the launch shape the bench's autotuner picks) and plain FP64 in the bench's
    shape.  Every system converges; 48 sampled systems are rechecked by the oracle (the refined ones by its
    FP64 residual, the FP64 ones against its iteration: equal sweep count, X within 1e-12)."""
    import torch
    ns, fs = synth.batch_shapes(4096, 64, 1024, 1.05, 2.0, synth.BASE_SEED + 2)
    As, Bs = [], []
    for k, (n, f) in enumerate(zip(ns, fs)):
        A, B, _ = synth.dominant_system(int(n), float(f), synth.system_seed(synth.BASE_SEED + 2, k))
        As.append(torch.from_numpy(A).cuda())
        Bs.append(torch.from_numpy(B[:, 0].copy()).cuda())
    bs = jac.BatchSolver(As, Bs, precision=prec, **shape)
    X = bs.solve_async(max_iter=5000, tol=1e-10)
    stats = bs.stats()
    if prec == "fp64":
        assert all(s.status == 0 for s in stats)
    else:
        assert all(s.status == 0 and s.rel_residual <= 1e-10 for s in stats)
    rng = np.random.default_rng(0)
    for k in rng.choice(4096, size=48, replace=False):
        # the oracle's inputs are regenerated on the host from the same seed
        A, B, _ = synth.dominant_system(int(ns[k]), float(fs[k]), synth.system_seed(synth.BASE_SEED + 2, int(k)))
        x = X[k].cpu().numpy()
        if prec == "fp64":
            ref = oracle.jacobi(A, B, max_iter=5000, tol=1e-10, norm=oracle.NORM_RESID)
            assert (stats[k].status, stats[k].sweeps) == (ref.status, ref.iters), k
            assert np.max(np.abs(x - ref.X[:, 0])) <= 1e-12 * np.max(np.abs(ref.X)), k
        else:
            _, rel = oracle.residual(A, B, x)
            assert rel <= 1e-10, (k, rel)


def test_one_call_batch_solve_equals_the_handle_path(jac):
    """jacobi_batch_solve (create, solve, records, release in one call, with the autotuner's launch shape
    for large batches: 4 rows per warp, 4 CTAs per SM, inner tolerance 2^-10) gives the handle path's
    results with that shape bit for bit, and its return value is the worst per-system outcome."""
    import torch
    systems = make_batch(23, 1, 400, 1.05, 2.0, seed=131)
    As, Bs = to_dev(systems)
    bs = jac.BatchSolver(As, Bs, precision="fp32_ir", rows_per_warp=4, ctas_per_sm=4, inner_rtol=2.0 ** -10)
    Xh = bs.solve_async(max_iter=5000, tol=1e-10)
    sh = bs.stats()
    Xs = [torch.empty(A.shape[0], dtype=torch.float64, device="cuda") for A in As]
    st, recs = jac.batch_solve(As, Bs, Xs, tol=1e-10, max_iter=5000, precision="fp32_ir")
    assert st == 0
    for k in range(len(As)):
        assert torch.equal(Xs[k], Xh[k]), k
        assert (recs[k].status, recs[k].sweeps, recs[k].outer_steps) == (sh[k].status, sh[k].sweeps, sh[k].outer_steps)
    # a cap that most systems hit: the call reports JACOBI_NOT_CONVERGED
    st, recs = jac.batch_solve(As, Bs, Xs, tol=1e-14, max_iter=2, precision="fp64")
    assert st == jac.NOT_CONVERGED and any(r.status == jac.NOT_CONVERGED for r in recs)
