"""Mixed-precision paths (FP32 / BF16 / E4M3 inner sweeps, FP64 refinement) on the GPU.

Parity of the iterates with the oracle is not expected (different arithmetic by design); what is pinned:
  * the narrow copies of A are bit-identical to the oracle's encoders (integer / byte work);
  * the returned X meets ||B - A X||_inf / ||B||_inf <= 1e-10, recomputed by the oracle in FP64;
  * the residual the kernel reports equals the oracle's residual of the returned X;
  * the error against the oracle's converged FP64 solution is within the residual bound.
"""
import numpy as np
import pytest

import oracle
import synth
from conftest import f64_narrowing_cases

pytestmark = pytest.mark.gpu

PRECS = ["fp32_ir", "bf16_ir", "fp8_ir"]


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


def qnorm(A):
    d = np.abs(np.diag(A))
    M = np.abs(A)
    np.fill_diagonal(M, 0.0)
    return float(np.max(M.sum(axis=1) / d))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n", [1, 33, 100, 1000])
def test_narrow_copy_bit_exact(jac, prec, n):
    A, B, _ = synth.dominant_system(n, 1.1, seed=40 + n)
    s = dev_solver(jac, A, B, precision=prec)
    got, scale = s.narrow()
    if prec == "fp32_ir":
        np.testing.assert_array_equal(got, oracle.offdiag_f32(A))
    elif prec == "bf16_ir":
        np.testing.assert_array_equal(got, oracle.offdiag_bf16(A))
    else:
        q, sc = oracle.offdiag_e4m3(A)
        np.testing.assert_array_equal(scale, sc)
        np.testing.assert_array_equal(got, q)


@pytest.mark.parametrize("prec", PRECS)
def test_narrow_copy_of_edge_values(jac, prec):
    """The setup's FP64 -> FP32 -> narrow rounding on ties, exponent carries, overflow to infinity, FP32
    subnormals and signed zeros (a matrix of such off-diagonals): codes identical to the oracle's.
    The E4M3 case uses the values that stay finite in FP32 (its row scale needs a finite maximum)."""
    x = f64_narrowing_cases(seed=3)
    if prec == "fp8_ir":
        with np.errstate(over="ignore"):
            x = x[np.isfinite(x.astype(np.float32))]
    n = int(np.ceil(np.sqrt(x.size))) + 1
    A = np.eye(n)
    off = ~np.eye(n, dtype=bool)
    A[off] = np.resize(x, off.sum())
    s = dev_solver(jac, A, np.ones((n, 1)), precision=prec)
    got, scale = s.narrow()
    if prec == "fp32_ir":
        np.testing.assert_array_equal(got.view(np.uint32), oracle.offdiag_f32(A).view(np.uint32))
    elif prec == "bf16_ir":
        np.testing.assert_array_equal(got, oracle.offdiag_bf16(A))
    else:
        q, sc = oracle.offdiag_e4m3(A)
        np.testing.assert_array_equal(scale.view(np.uint32), sc.view(np.uint32))
        np.testing.assert_array_equal(got, q)


@pytest.mark.parametrize("prec", ["bf16_ir", "fp32_ir"])
@pytest.mark.parametrize("n", [1, 2, 33, 100, 1000, 1537])
def test_first_solve_writes_the_narrow_copy(jac, prec, n):
    """BF16 / FP32 inner sweeps: the first inner sweep of a handle's first solve streams FP64 A, writes the
    narrow copy and sweeps over the rounded values.  The copy it leaves is bit-identical to the oracle's
    encoder (ragged last chunk, diagonal, row padding); later solves read it instead."""
    A, B, _ = synth.dominant_system(n, 1.1, seed=70 + n)
    s = dev_solver(jac, A, B, precision=prec)
    X, st = s.solve(max_iter=5000, tol=1e-10)
    kinds = [k for k, _, _ in s.trace()]
    assert kinds.count(jac.binding.PHASE_NARROW_INNER) == 1 and kinds[1] == jac.binding.PHASE_NARROW_INNER
    _, rel = oracle.residual(A, B, X.cpu().numpy())
    assert st.status == 0 and rel <= 1e-10
    got, _ = s.narrow()
    want = oracle.offdiag_f32(A) if prec == "fp32_ir" else oracle.offdiag_bf16(A)
    np.testing.assert_array_equal(got.view(np.uint16 if prec == "bf16_ir" else np.uint32),
                                  want.view(np.uint16 if prec == "bf16_ir" else np.uint32))
    # a second solve on the handle sweeps the stored copy; so does a handle whose copy was read out first
    # (setup's own narrow pass): the two solves are then the same computation, bit for bit
    X2, st2 = s.solve(max_iter=5000, tol=1e-10)
    assert jac.binding.PHASE_NARROW_INNER not in [k for k, _, _ in s.trace()]
    t = dev_solver(jac, A, B, precision=prec)
    t.narrow()
    X3, st3 = t.solve(max_iter=5000, tol=1e-10)
    assert jac.binding.PHASE_NARROW_INNER not in [k for k, _, _ in t.trace()]
    assert (st2.sweeps, st2.outer_steps) == (st3.sweeps, st3.outer_steps)
    np.testing.assert_array_equal(X2.cpu().numpy(), X3.cpu().numpy())


@pytest.mark.parametrize("prec", ["bf16_ir", "fp32_ir"])
def test_first_solve_writes_the_narrow_copy_of_edge_values(jac, prec):
    """The fused first sweep rounds ties, exponent carries, overflows and FP32 subnormals as the setup pass
    does; the solve itself ends NONFINITE (the matrix is not dominant), after the copy is complete."""
    import torch
    x = f64_narrowing_cases(seed=4)
    n = int(np.ceil(np.sqrt(x.size))) + 1
    A = np.eye(n)
    off = ~np.eye(n, dtype=bool)
    A[off] = np.resize(x, off.sum())
    s = dev_solver(jac, A, np.ones((n, 1)), precision=prec)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    s.solve_async(None, 50, 1e-10, out)
    s.last_stats()
    assert jac.binding.PHASE_NARROW_INNER in [k for k, _, _ in s.trace()]
    got, _ = s.narrow()
    want = oracle.offdiag_f32(A) if prec == "fp32_ir" else oracle.offdiag_bf16(A)
    np.testing.assert_array_equal(got.view(np.uint16 if prec == "bf16_ir" else np.uint32),
                                  want.view(np.uint16 if prec == "bf16_ir" else np.uint32))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("gen,n,f", [("dom", 1, 1.25), ("dom", 33, 1.25), ("dom", 512, 1.25), ("dom", 4096, 1.05),
                                     ("hard", 300, 1.25), ("hard", 2000, 1.1)])
def test_refinement_reaches_target(jac, prec, gen, n, f):
    make = synth.dominant_system if gen == "dom" else synth.hard_system
    A, B, Xs = make(n, f, seed=50 + n)
    target = 1e-10
    s = dev_solver(jac, A, B, precision=prec)
    X, st = s.solve(max_iter=5000, tol=target)
    Xh = X.cpu().numpy()
    _, rel = oracle.residual(A, B, Xh)
    assert st.status == 0 and rel <= target, (st.as_dict(), rel)
    assert abs(st.rel_residual - rel) <= 1e-13 + 1e-3 * rel
    q = qnorm(A)
    ref = oracle.jacobi(A, B, max_iter=20000, tol=1e-14)
    err = np.max(np.abs(Xh[:, None] - ref.X)) / np.max(np.abs(ref.X))
    assert err <= 2 * target * (1 + q) / (1 - q) + 1e-13, err
    print(f"{prec} {gen} n={n}: outer={st.outer_steps} inner={st.sweeps} residual={rel:.2e} err={err:.2e}")


@pytest.mark.parametrize("prec", PRECS)
def test_full_size_single_system(jac, prec):
    """n = 16384, f = 1.05: relative residual <= 1e-10 recomputed on the CPU."""
    A, B, _ = synth.dominant_system(16384, 1.05, seed=synth.BASE_SEED + 1)
    s = dev_solver(jac, A, B, precision=prec)
    X, st = s.solve(max_iter=5000, tol=1e-10)
    _, rel = oracle.residual(A, B, X.cpu().numpy())
    assert st.status == 0 and rel <= 1e-10, (st.as_dict(), rel)


def test_nonzero_start_vector(jac):
    import torch
    A, B, Xs = synth.dominant_system(700, 1.25, seed=61)
    X0 = Xs[:, 0] + 1e-3 * np.linspace(-1, 1, 700)
    s = dev_solver(jac, A, B, precision="bf16_ir")
    X, st = s.solve(X0=torch.from_numpy(X0).cuda(), max_iter=500, tol=1e-10)
    _, rel = oracle.residual(A, B, X.cpu().numpy())
    assert st.status == 0 and rel <= 1e-10
    # a start vector that already meets the target returns after one residual evaluation
    X2, st2 = s.solve(X0=X.clone(), max_iter=500, tol=1e-10)
    assert st2.outer_steps == 1 and st2.sweeps == 0
    assert torch.equal(X2, X)


@pytest.mark.parametrize("prec", ["fp64", "fp32_ir", "bf16_ir", "fp8_ir"])
def test_zero_right_hand_side(jac, prec):
    """B = 0, the degenerate case (the solution is X = 0).  The max-norm stop (FP64) sees no change in the
    first sweep and stops there, as the oracle does.  The relative-residual stop of the refinement is
    ||B - A X|| / ||B|| = 0 / 0: reported as JACOBI_ERR_NONFINITE at the first residual with X left at the
    zero start vector, as the oracle's residual-norm stop reports it."""
    import torch
    n = 300
    A, _, _ = synth.dominant_system(n, 1.2, seed=71)
    B = np.zeros((n, 1))
    s = dev_solver(jac, A, B, precision=prec)
    tol = 1e-12 if prec == "fp64" else 1e-10
    out = s.solve_async(None, 100, tol)
    st = s.last_stats()
    ref = oracle.jacobi(A, B, max_iter=100, tol=tol, norm=oracle.NORM_INF if prec == "fp64" else oracle.NORM_RESID)
    assert st.status == ref.status, (st.status, ref.status)
    assert int(torch.count_nonzero(out)) == 0
    if prec == "fp64":
        assert st.status == 0 and st.sweeps == ref.iters == 1
    else:
        assert st.status == jac.ERR_NONFINITE


def test_outer_cap_reports_not_converged(jac):
    A, B, _ = synth.hard_system(500, 1.1, seed=62)
    s = dev_solver(jac, A, B, precision="bf16_ir", max_outer=2)
    X, st = s.solve(max_iter=5000, tol=1e-14)
    assert st.status == jac.NOT_CONVERGED and st.outer_steps == 2
    _, rel = oracle.residual(A, B, X.cpu().numpy())
    assert abs(st.rel_residual - rel) <= 1e-13 + 1e-3 * rel


def test_device_residual_entry_point(jac):
    import torch
    A, B, Xs = synth.dominant_system(777, 1.1, seed=63)
    s = dev_solver(jac, A, B)
    x = torch.from_numpy(Xs[:, 0] + 1e-6).cuda()
    _, rel = oracle.residual(A, B, x.cpu().numpy())
    assert abs(s.residual(x) - rel) <= 1e-14 + 1e-9 * rel


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("gen,n,f", [("dom", 777, 1.1), ("hard", 1500, 1.1), ("dom", 4096, 1.05)])
def test_split_float_residual_reaches_target(jac, prec, gen, n, f):
    make = synth.dominant_system if gen == "dom" else synth.hard_system
    A, B, _ = make(n, f, seed=70 + n)
    s = dev_solver(jac, A, B, precision=prec, split_residual=True)
    X, st = s.solve(max_iter=5000, tol=1e-10)
    _, rel = oracle.residual(A, B, X.cpu().numpy())
    assert st.status == 0 and rel <= 1e-10, (st.as_dict(), rel)
    assert abs(st.rel_residual - rel) <= 5e-13 + 1e-3 * rel


def test_split_float_residual_accuracy_with_wild_row_scales(jac):
    """One residual evaluation of a given X0 (max_outer = 1): the split-float residual equals the oracle's
    FP64 residual to ~1e-15 of ||A|| ||X||, on rows scaled by powers of two from 2^-300 to 2^+300 and an
    X0 whose entries span many magnitudes."""
    import torch
    n = 1000
    A, B, Xs = synth.dominant_system(n, 1.3, seed=91)
    rng = np.random.default_rng(2)
    scale = 2.0 ** rng.integers(-300, 300, n)
    A = A * scale[:, None]
    B = B * scale[:, None]
    X0 = Xs[:, 0] * (1 + 1e-6 * rng.standard_normal(n))
    X0[::7] *= 1e3
    s = dev_solver(jac, A, B, precision="bf16_ir", split_residual=True, max_outer=1)
    _, st = s.solve(X0=torch.from_numpy(X0).cuda(), max_iter=10, tol=1e-300)
    assert st.outer_steps == 1 and st.sweeps == 0
    _, rel = oracle.residual(A, B, X0)
    assert abs(st.rel_residual - rel) <= 1e-12 * rel, (st.rel_residual, rel)


@pytest.mark.parametrize("prec", ["fp32_ir", "bf16_ir", "fp8_ir"])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_resident_inputs_match_device_inputs(jac, prec, pinned):
    """A and B in host memory (pinned or pageable), copied into the workspace by the setup: the narrow
    copy and the solution are identical, bit for bit, to those of the same system given in device
    memory."""
    import torch
    n = 1000
    A, B, _ = synth.dominant_system(n, 1.1, seed=95)
    Ah = torch.from_numpy(A)
    Bh = torch.from_numpy(B[:, 0].copy())
    if pinned:
        Ah, Bh = Ah.pin_memory(), Bh.pin_memory()
    sh = jac.DeviceSolver(Ah, Bh, precision=prec, device=torch.device("cuda", 0))
    sd = dev_solver(jac, A, B, precision=prec)
    nh, sch = sh.narrow()
    nd, scd = sd.narrow()
    np.testing.assert_array_equal(nh, nd)
    np.testing.assert_array_equal(sch, scd)
    Xh, sth = sh.solve(max_iter=5000, tol=1e-10)
    Xd, std = sd.solve(max_iter=5000, tol=1e-10)
    assert torch.equal(Xh, Xd) and (sth.sweeps, sth.outer_steps) == (std.sweeps, std.outer_steps)
    _, rel = oracle.residual(A, B, Xh.cpu().numpy())
    assert sth.status == 0 and rel <= 1e-10
