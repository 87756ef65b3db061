"""Symmetric A stored once (JACOBI_FLAG_SYMMETRIC): BF16 / FP32 inner sweeps over the packed upper tiles.

* One inner sweep: with one outer step and one inner sweep, X = c1 - f (Q c1), where Q holds the oracle's
  BF16 (or FP32) values of the off-diagonal part of A, c1 = fl32(b / a_ii) and f = fl32(1 / a_ii); the kernel
  accumulates in FP32, so the tolerance is FP32 rounding over n terms.  Sizes cover one tile, a ragged last
  tile row and column, and several tiles.
* Refinement: ||B - A X||_inf / ||B||_inf <= 1e-10 recomputed by the oracle, and X within the bound that two
  solutions of residual 1e-10 and 1e-12 obey (strict dominance: ||A^-1||_inf <= 1 / min_i (|a_ii| -
  sum_{j!=i} |a_ij|)) of the oracle's FP64 Jacobi solution and of the full-storage refinement's X.
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


def dev(A, b):
    import torch
    return torch.from_numpy(A).cuda(), torch.from_numpy(np.ascontiguousarray(b)).cuda()


def narrow_values(A, prec):
    if prec == "bf16_ir":
        return (oracle.offdiag_bf16(A).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return oracle.offdiag_f32(A).astype(np.float64)


@pytest.mark.parametrize("prec", ["bf16_ir", "fp32_ir"])
@pytest.mark.parametrize("n", [1, 100, 128, 300, 1000])
def test_one_symmetric_inner_sweep(jac, n, prec):
    A, B, _ = synth.symmetric_system(n, 1.1, seed=40 + n)
    b = B[:, 0].copy()
    At, bt = dev(A, b)
    s = jac.DeviceSolver(At, bt, precision=prec, symmetric=True, max_outer=2, max_inner=1)
    X, st = s.solve(max_iter=10, tol=1e-300)
    assert st.outer_steps == 2 and st.sweeps == 1
    got = X.cpu().numpy()
    rinv = 1.0 / np.diag(A)
    c1 = (b * rinv).astype(np.float32).astype(np.float64)
    f = rinv.astype(np.float32).astype(np.float64)
    Q = narrow_values(A, prec)
    want = c1 - f * (Q @ c1)
    scale = np.abs(f) * (np.abs(Q) @ np.abs(c1))
    assert np.all(np.abs(got - want) <= 2e-6 * scale + 1e-12), np.max(np.abs(got - want) / (scale + 1e-300))


@pytest.mark.parametrize("prec", ["bf16_ir", "fp32_ir"])
@pytest.mark.parametrize("n,f,gen", [(5, 1.2, "dom"), (129, 1.05, "dom"), (640, 1.1, "dom"), (2049, 1.05, "dom"),
                                     (700, 1.3, "hard")])
def test_symmetric_refinement_reaches_target(jac, n, f, gen, prec):
    if gen == "dom":
        A, B, Xs = synth.symmetric_system(n, f, seed=60 + n)
    else:  # the paper-shaped generator made symmetric: positive entries, rho(T) close to 1/f
        A, B, Xs = synth.hard_system(n, f, seed=60 + n)
        A = np.triu(A, 1)
        A = A + A.T
        A[np.arange(n), np.arange(n)] = f * A.sum(axis=1)
        B = A @ Xs
    b = B[:, 0].copy()
    At, bt = dev(A, b)
    s = jac.DeviceSolver(At, bt, precision=prec, symmetric=True)
    X, st = s.solve(max_iter=5000, tol=1e-10)
    Xh = X.cpu().numpy()
    _, rel = oracle.residual(A, B, Xh)
    assert st.status == 0 and rel <= 1e-10, (st.as_dict(), rel)
    assert abs(st.rel_residual - rel) <= 1e-13 + 1e-3 * rel
    d = np.abs(np.diag(A))
    margin = np.min(d - (np.abs(A).sum(axis=1) - d))
    bound = (1e-10 + 2e-12) * np.max(np.abs(b)) / margin
    ref = oracle.jacobi(A, B, max_iter=20000, tol=1e-12, norm=oracle.NORM_RESID)
    assert ref.status == oracle.OK
    assert np.max(np.abs(Xh - ref.X[:, 0])) <= bound
    full = jac.DeviceSolver(At, bt, precision=prec)
    Xf, stf = full.solve(max_iter=5000, tol=1e-10)
    assert stf.status == 0
    assert np.max(np.abs(Xh - Xf.cpu().numpy())) <= 2 * bound


def test_symmetric_flag_combinations(jac):
    import torch
    A, B, _ = synth.symmetric_system(64, 1.2, seed=3, nrhs=2)
    At = torch.from_numpy(A).cuda()
    b = torch.from_numpy(np.ascontiguousarray(B[:, 0])).cuda()
    for prec in ("fp64", "fp8_ir"):
        with pytest.raises(jac.JacobiError) as e:
            jac.DeviceSolver(At, b, precision=prec, symmetric=True)
        assert e.value.status == jac.ERR_UNSUPPORTED
    with pytest.raises(jac.JacobiError) as e:
        jac.DeviceSolver(At, b, precision="bf16_ir", symmetric=True, split_residual=True)
    assert e.value.status == jac.ERR_INVALID_ARG
    s = jac.DeviceSolver(At, b, precision="bf16_ir", symmetric=True)
    X, st = s.solve(max_iter=100, tol=1e-10)
    kinds = [k for k, _, _ in s.trace() if k != 5]  # 5: the stream idle while the host decides
    assert st.status == 0 and kinds[0] == 2 and 3 in kinds  # zero-start residual, then inner sweeps
