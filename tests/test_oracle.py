"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Every check compares the oracle with something other than itself: hand-derived iterates, a textbook
system with a known solution, Gaussian elimination and scipy's LU solver, the a-priori and a-posteriori
contraction bounds, the planted solution, the residual identity of Section 2's component update, the
closed-form spectral radius of the paper-shaped generator, and torch's BF16 / E4M3 conversions.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import f64_narrowing_cases, read_golden


def tnorm_inf(A):
    """||T||_inf of T = D^-1 (L + U) straight from A: max_i sum_{j!=i} |a_ij| / |a_ii|."""
    d = np.abs(np.diag(A))
    off = np.abs(A).sum(axis=1) - d
    return float(np.max(off / d))


# ---------------------------------------------------------------- hand-derived and textbook fixtures

def test_golden_2x2_iterates():
    g = read_golden("jacobi_2x2.txt")
    A = np.array(g["A"]).reshape(2, 2)
    B = np.array(g["B"])
    res = oracle.jacobi(A, B, max_iter=4, tol=1e-300, trace=True)
    assert res.status == oracle.NOT_CONVERGED and res.iters == 4
    for k, want in g["iters"].items():
        np.testing.assert_allclose(res.trace[k - 1][:, 0], want, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(res.X[:, 0], res.trace[3][:, 0])
    full = oracle.jacobi(A, B, max_iter=200, tol=1e-15)
    assert full.status == oracle.OK
    np.testing.assert_allclose(full.X[:, 0], g["SOLUTION"], rtol=0, atol=1e-14)
    # by hand: delta_2 = 0.1 and delta_3 = 0.04, so tol = 0.05 stops at k = 3 and returns the NEW
    # iterate X^3 (Section 2 algorithm: "return X" after the test on X - X^t)
    stop = oracle.jacobi(A, B, max_iter=10, tol=0.05)
    assert stop.status == oracle.OK and stop.iters == 3
    np.testing.assert_allclose(stop.X[:, 0], g["iters"][3], rtol=0, atol=1e-15)
    assert abs(stop.delta - 0.04) < 1e-15


def test_golden_4x4_textbook():
    g = read_golden("jacobi_4x4_textbook.txt")
    A = np.array(g["A"]).reshape(4, 4)
    B = np.array(g["B"])
    first = oracle.jacobi(A, B, max_iter=1, tol=1e-300)
    np.testing.assert_allclose(first.X[:, 0], g["iters"][1], rtol=0, atol=1e-15)
    res = oracle.jacobi(A, B, max_iter=500, tol=1e-13)
    assert res.status == oracle.OK
    np.testing.assert_allclose(res.X[:, 0], g["SOLUTION"], rtol=0, atol=1e-12)


def test_split_2x2_by_hand():
    A = np.array([[4.0, 1.0], [2.0, 5.0]])
    st, T, C = oracle.split(A, [1.0, 2.0])
    assert st == oracle.OK
    np.testing.assert_array_equal(T, [[0.0, -0.25], [-0.4, 0.0]])
    np.testing.assert_array_equal(C[:, 0], [0.25, 0.4])


# ------------------------------------------------------------------- direct solver (Gaussian elim.)

@pytest.mark.parametrize("n", [1, 2, 3, 17, 64])
def test_ge_recovers_planted_and_matches_scipy(n):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(n)
    A = rng.uniform(-1, 1, (n, n)) + np.eye(n) * 0.5   # general (not dominant) matrix
    Xs = rng.uniform(-1, 1, (n, 2))
    B = A @ Xs
    st, X = oracle.ge(A, B)
    assert st == oracle.OK
    cond = np.linalg.cond(A)
    np.testing.assert_allclose(X, Xs, rtol=0, atol=1e-14 * cond * n)
    np.testing.assert_allclose(X, scipy_linalg.solve(A, B), rtol=0, atol=1e-14 * cond * n)


def test_ge_singular():
    A = np.array([[1.0, 2.0], [2.0, 4.0]])
    st, _ = oracle.ge(A, [1.0, 1.0])
    assert st == oracle.ZERO_DIAGONAL


# ------------------------------------------------------------- Jacobi: converged value and bounds

@pytest.mark.parametrize("n,f,gen", [(8, 1.25, "dom"), (33, 1.1, "dom"), (64, 1.25, "hard"),
                                     (50, 2.0, "hard")])
def test_jacobi_converges_to_ge(n, f, gen):
    make = synth.dominant_system if gen == "dom" else synth.hard_system
    A, B, Xs = make(n, f, seed=100 + n)
    q = tnorm_inf(A)
    assert q < 1
    tol = 1e-13
    res = oracle.jacobi(A, B, max_iter=5000, tol=tol)
    assert res.status == oracle.OK
    st, Xge = oracle.ge(A, B)
    assert st == oracle.OK
    # a-posteriori bound ||X^k - X*|| <= q/(1-q) ||X^k - X^(k-1)||, plus rounding
    bound = q / (1 - q) * res.delta + 1e-14
    assert np.max(np.abs(res.X - Xge)) <= bound
    assert np.max(np.abs(res.X - Xs)) <= bound


@pytest.mark.parametrize("gen,f", [("dom", 1.25), ("dom", 1.05), ("hard", 1.25)])
def test_a_priori_and_a_posteriori_bounds(gen, f):
    n = 40
    make = synth.dominant_system if gen == "dom" else synth.hard_system
    A, B, Xs = make(n, f, seed=7)
    q = tnorm_inf(A)
    assert abs(q - 1 / f) < 1e-12
    X0 = np.linspace(-2, 3, n)[:, None]
    res = oracle.jacobi(A, B, X0=X0, max_iter=60, tol=1e-300, trace=True)
    e0 = np.max(np.abs(X0 - Xs))
    prev = X0
    for k in range(1, res.iters + 1):
        Xk = res.trace[k - 1]
        err = np.max(np.abs(Xk - Xs))
        assert err <= q ** k * e0 * (1 + 1e-12) + 1e-14, k                  # a-priori
        assert err <= q / (1 - q) * np.max(np.abs(Xk - prev)) + 1e-14, k    # a-posteriori
        prev = Xk


def test_planted_solution_recovery():
    A, B, Xs = synth.dominant_system(200, 1.25, seed=3)
    res = oracle.jacobi(A, B, max_iter=2000, tol=1e-12)
    assert res.status == oracle.OK
    q = tnorm_inf(A)
    assert np.max(np.abs(res.X - Xs)) <= q / (1 - q) * 1e-12 + 1e-14


def test_diagonal_matrix_one_sweep():
    d = np.array([2.0, -3.0, 7.0, 0.1, 1e3])
    A = np.diag(d)
    B = np.array([1.0, 1.0, -2.0, 5.0, 3.0])
    res = oracle.jacobi(A, B, max_iter=10, tol=1e-12, trace=True)
    # T = 0 so X^1 = C = B / d (one correctly rounded division each) and X^2 = X^1
    np.testing.assert_array_equal(res.trace[0][:, 0], B / d)
    assert res.status == oracle.OK and res.iters == 2 and res.delta == 0.0
    res1 = oracle.jacobi(A, B, X0=B / d, max_iter=10, tol=1e-12)
    assert res1.iters == 1 and res1.delta == 0.0


def test_residual_identity():
    """b_i - sum_j a_ij x_j^(k) = a_ii (x_i^(k+1) - x_i^(k)) for every k (Section 2 update rearranged)."""
    A, B, _ = synth.dominant_system(30, 1.25, seed=11)
    res = oracle.jacobi(A, B, max_iter=8, tol=1e-300, trace=True)
    d = np.diag(A)[:, None]
    scale = np.abs(A).sum(axis=1, keepdims=True) * 2
    for k in range(1, res.iters):
        R, _ = oracle.residual(A, B, res.trace[k - 1])
        want = d * (res.trace[k] - res.trace[k - 1])
        assert np.all(np.abs(R - want) <= 1e-14 * scale)


def test_residual_matches_numpy():
    rng = np.random.default_rng(5)
    A = rng.uniform(-1, 1, (37, 37))
    B = rng.uniform(-1, 1, (37, 3))
    X = rng.uniform(-1, 1, (37, 3))
    R, rel = oracle.residual(A, B, X)
    want = B - A @ X
    np.testing.assert_allclose(R, want, rtol=0, atol=1e-14)
    want_rel = max(np.max(np.abs(want[:, c])) / np.max(np.abs(B[:, c])) for c in range(3))
    assert abs(rel - want_rel) <= 1e-14 * want_rel


def test_hard_generator_rate_is_one_over_f():
    """Paper-shaped generator: T = -(1/f) S with S row-stochastic, so the error contracts by 1/f."""
    f = 1.25
    A, B, Xs = synth.hard_system(64, f, seed=2)
    _, T, _ = oracle.split(A, B)
    np.testing.assert_allclose(T.sum(axis=1), -1 / f, rtol=1e-14)
    assert abs(max(abs(np.linalg.eigvals(T))) - 1 / f) < 1e-10
    res = oracle.jacobi(A, B, max_iter=80, tol=1e-300, trace=True)
    errs = [np.max(np.abs(res.trace[k] - Xs)) for k in range(res.iters)]
    ratio = errs[60] / errs[59]
    assert abs(ratio - 1 / f) < 1e-3
    # predicted sweep count to reach tol from ||X0 - X*|| (X0 = 0): ln(tol / e0) / ln(1/f) + O(1)
    tol = 1e-10
    full = oracle.jacobi(A, B, max_iter=5000, tol=tol)
    pred = math.log(tol / np.max(np.abs(Xs))) / math.log(1 / f)
    assert abs(full.iters - pred) < 0.15 * pred


def test_residual_rows_equal_the_full_residual():
    A, B, Xs = synth.dominant_system(150, 1.1, seed=17, nrhs=4)
    X = Xs + 1e-7 * np.sin(np.arange(Xs.size)).reshape(Xs.shape)
    R, _ = oracle.residual(A, B, X)
    rows = np.array([149, 0, 77, 77, 3])
    np.testing.assert_array_equal(oracle.residual_rows(A, B, X, rows), R[rows])
    with pytest.raises(ValueError):
        oracle.residual_rows(A, B, X, [150])


def test_split_fixed_point():
    A, B, Xs = synth.dominant_system(50, 1.25, seed=4, nrhs=2)
    st, T, C = oracle.split(A, B)
    assert st == oracle.OK
    assert np.all(np.diag(T) == 0)
    np.testing.assert_allclose(T @ Xs + C, Xs, rtol=0, atol=1e-14)
    i, j = 3, 17
    assert T[i, j] == -A[i, j] / A[i, i]


# ------------------------------------------------------------------------------ control flow

def test_strict_stopping_test():
    A = np.array([[1.0]])
    B = np.array([0.5])
    r = oracle.jacobi(A, B, max_iter=5, tol=0.5)       # delta_1 = 0.5 is not < 0.5
    assert r.status == oracle.OK and r.iters == 2 and r.delta == 0.0
    r = oracle.jacobi(A, B, max_iter=5, tol=0.5000001)
    assert r.status == oracle.OK and r.iters == 1 and r.delta == 0.5


def test_iteration_cap_returns_last_iterate():
    A, B, _ = synth.hard_system(20, 1.05, seed=9)
    r = oracle.jacobi(A, B, max_iter=3, tol=1e-15, trace=True)
    assert r.status == oracle.NOT_CONVERGED and r.iters == 3
    np.testing.assert_array_equal(r.X, r.trace[2])
    assert r.delta == np.max(np.abs(r.trace[2] - r.trace[1]))


def test_error_statuses():
    A = np.array([[1.0, 0.1], [0.2, 0.0]])
    assert oracle.jacobi(A, [1.0, 1.0]).status == oracle.ZERO_DIAGONAL
    A[1, 1] = np.nan
    assert oracle.jacobi(A, [1.0, 1.0]).status == oracle.NONFINITE
    A[1, 1] = np.inf
    assert oracle.jacobi(A, [1.0, 1.0]).status == oracle.NONFINITE
    good = np.eye(2)
    assert oracle.jacobi(good, [1.0, 1.0], max_iter=0).status == oracle.INVALID_ARG
    assert oracle.jacobi(good, [1.0, 1.0], tol=0.0).status == oracle.INVALID_ARG
    assert oracle.jacobi(good, [1.0, 1.0], tol=float("nan")).status == oracle.INVALID_ARG
    assert oracle.jacobi(good, [1.0, 1.0], norm=7).status == oracle.INVALID_ARG


def test_divergence_reports_nonfinite():
    A = np.array([[1.0, 10.0], [10.0, 1.0]])              # rho(T) = 10: iterates overflow
    r = oracle.jacobi(A, [1.0, 1.0], max_iter=2000, tol=1e-12)
    assert r.status == oracle.NONFINITE
    assert 300 < r.iters < 320


def test_euclidean_norm_mode():
    d = np.array([2.0, 4.0, 5.0])
    B = np.array([1.0, -2.0, 3.0])
    r = oracle.jacobi(np.diag(d), B, max_iter=1, tol=10.0, norm=oracle.NORM_2)
    assert r.iters == 1 and abs(r.delta - np.linalg.norm(B / d)) <= 1e-16


def test_residual_norm_mode_is_relative_residual_of_previous_iterate():
    A, B, _ = synth.dominant_system(25, 1.1, seed=13)
    full = oracle.jacobi(A, B, max_iter=6, tol=1e-300, norm=oracle.NORM_RESID, trace=True)
    for k in range(2, full.iters + 1):
        part = oracle.jacobi(A, B, max_iter=k, tol=1e-300, norm=oracle.NORM_RESID)
        _, rel = oracle.residual(A, B, full.trace[k - 2])
        # both sides are normalised by ||B||_inf; the residual itself is a cancellation of O(1) terms,
        # so the rounding error is absolute in these units (~ n * eps * ||A|| ||X|| / ||B||)
        assert abs(part.delta - rel) <= 1e-14


def test_multi_rhs_columns_are_independent():
    A, B, _ = synth.dominant_system(20, 1.25, seed=21, nrhs=3)
    multi = oracle.jacobi(A, B, max_iter=5, tol=1e-300)
    for c in range(3):
        one = oracle.jacobi(A, B[:, c], max_iter=5, tol=1e-300)
        np.testing.assert_array_equal(multi.X[:, c], one.X[:, 0])


def _per_column_changes(trace, X0, norm):
    """Per sweep k and column c: the Euclidean length of X^(k) - X^(k-1) (numpy's norm), from a trace."""
    prev = np.concatenate([X0[None], trace[:-1]])
    if norm == oracle.NORM_2:
        return np.linalg.norm(trace - prev, axis=1)
    raise ValueError(norm)


@pytest.mark.parametrize("scales", [(1.0, 1.0, 1.0), (2.0 ** -20, 1.0, 2.0 ** 20), (2.0 ** 30, 2.0 ** -30, 1.0)])
def test_euclidean_norm_over_several_columns_is_the_largest_column_length(scales):
    # Section 2 measures the change of one system by its Euclidean length; with several right-hand sides
    # each column is its own system, so the decisive value is the largest column length.  Equal columns
    # tell this apart from the length of all columns together (sqrt(3) times larger); columns of very
    # different magnitude tell it apart from the first, last or smallest column's length.
    A, B0, _ = synth.dominant_system(24, 1.1, seed=31, nrhs=3)
    if scales[0] == scales[1] == scales[2]:
        B0 = np.repeat(B0[:, :1], 3, axis=1)
    B = B0 * np.array(scales)
    X0 = np.zeros_like(B)
    full = oracle.jacobi(A, B, max_iter=60, tol=1e-300, norm=oracle.NORM_2, trace=True)
    per_col = _per_column_changes(full.trace, X0, oracle.NORM_2)        # (k, c)
    for k in (1, 2, 5, 17):
        part = oracle.jacobi(A, B, max_iter=k, tol=1e-300, norm=oracle.NORM_2)
        want = per_col[k - 1].max()
        assert abs(part.delta - want) <= 1e-14 * want, (k, part.delta, want)
    # the stop: the first sweep whose largest column length is below tol (strict)
    tol = float(np.sort(per_col.max(axis=1))[::-1][12]) * 1.0000001
    first = int(np.argmax(per_col.max(axis=1) < tol)) + 1
    stop = oracle.jacobi(A, B, max_iter=60, tol=tol, norm=oracle.NORM_2)
    assert stop.status == oracle.OK and stop.iters == first
    np.testing.assert_array_equal(stop.X, full.trace[first - 1])
    if scales[0] == scales[1] == scales[2]:
        total = np.sqrt((per_col ** 2).sum(axis=1))
        assert np.all(total > 1.7 * per_col.max(axis=1))               # the reading is distinguishable


def test_residual_norm_over_several_columns_is_the_worst_relative_column():
    # The residual-norm stop of the previous iterate, per column: ||b_c - A x_c^(k-1)||_inf / ||b_c||_inf
    # (each column its own system), and the largest of these decides.  Column 2 has the smallest right-hand
    # side and a start far from its solution, so its relative residual leads; pooling the residuals and
    # right-hand sides of all columns would give a value about a million times smaller.
    A, B, _ = synth.dominant_system(30, 1.2, seed=33, nrhs=3)
    B = B * np.array([2.0 ** 20, 1.0, 2.0 ** -20])
    X0 = np.zeros_like(B)
    X0[:, 2] = 2.0 ** -10
    full = oracle.jacobi(A, B, X0=X0, max_iter=8, tol=1e-300, norm=oracle.NORM_RESID, trace=True)
    prev = np.concatenate([X0[None], full.trace[:-1]])
    for k in range(1, full.iters + 1):
        part = oracle.jacobi(A, B, X0=X0, max_iter=k, tol=1e-300, norm=oracle.NORM_RESID)
        rels = [oracle.residual(A, B[:, c], prev[k - 1][:, c])[1] for c in range(3)]
        assert int(np.argmax(rels)) == 2
        want = max(rels)
        assert abs(part.delta - want) <= 1e-14 * want, (k, part.delta, rels)
        R, _ = oracle.residual(A, B, prev[k - 1])
        pooled = np.abs(R).max() / np.abs(B).max()
        assert pooled < 1e-3 * want                                    # the pooled reading differs


def test_thread_count_does_not_change_results():
    A, B, _ = synth.hard_system(97, 1.1, seed=5, nrhs=2)
    a = oracle.jacobi(A, B, max_iter=40, tol=1e-300, nthreads=1)
    b = oracle.jacobi(A, B, max_iter=40, tol=1e-300, nthreads=4)
    np.testing.assert_array_equal(a.X, b.X)


# ------------------------------------------------------------------ narrow encodings of T's factors

def _f32_cases():
    rng = np.random.default_rng(0)
    vals = np.concatenate([
        rng.standard_normal(20000).astype(np.float32),
        (rng.uniform(-1, 1, 20000) * 2.0 ** rng.integers(-140, 120, 20000)).astype(np.float32),
        np.array([0.0, -0.0, 1.0, -1.0, 3.4e38, -3.4e38, 1e-45, 1.00390625, 1.01171875, 1.0078125,
                  np.float32(1) + np.float32(2 ** -8), 65504.0], dtype=np.float32),
    ])
    # exact BF16 ties: mantissa bits below the kept 7 exactly at the half-way point
    ties = (np.arange(1000, dtype=np.uint32) << 16) | np.uint32(0x3F808000)
    return np.concatenate([vals, ties.view(np.float32)])


def test_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    x = _f32_cases()
    want = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    got = np.array([oracle.bf16_from_f32(v) for v in x], dtype=np.uint16)
    np.testing.assert_array_equal(got, want)


def test_e4m3_matches_torch_in_range_and_saturates():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-448, 448, 20000), rng.uniform(-1, 1, 5000) * 2.0 ** -7,
                        [0.0, 448.0, -448.0, 2.0 ** -9, 2.0 ** -10, 0.5 * 2.0 ** -9, 1.5 * 2.0 ** -9,
                         1.0625, 1.1875, 240.0, 232.0, 248.0]]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    got = np.array([oracle.e4m3_from_f32(v) for v in x], dtype=np.uint8)
    np.testing.assert_array_equal(got, want)
    assert oracle.e4m3_from_f32(1000.0) == 0x7E and oracle.e4m3_from_f32(-1e30) == 0xFE
    assert oracle.e4m3_from_f32(460.0) == 0x7E


def test_offdiag_encodings():
    torch = pytest.importorskip("torch")
    A, _, _ = synth.dominant_system(37, 1.1, seed=8)
    f32 = oracle.offdiag_f32(A)
    off = A.copy()
    np.fill_diagonal(off, 0.0)
    np.testing.assert_array_equal(f32, off.astype(np.float32))
    bf = oracle.offdiag_bf16(A)
    want = torch.from_numpy(off.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy()
    np.testing.assert_array_equal(bf, want.view(np.uint16))
    q, s = oracle.offdiag_e4m3(A)
    m = np.abs(off.astype(np.float32)).max(axis=1).astype(np.float64)
    # the row scale is the smallest power of two s with m <= 448 s
    mant, _ = np.frexp(s.astype(np.float64))
    assert np.all(mant == 0.5)                                   # powers of two
    assert np.all(m <= 448.0 * s) and np.all(m > 224.0 * s)      # and the smallest such
    assert np.all(np.diag(q) == 0)
    scaled = (off.astype(np.float32) / s[:, None]).astype(np.float32)
    want_q = torch.from_numpy(scaled).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    np.testing.assert_array_equal(q, want_q)
    # the row maximum, in (224, 448] after scaling, is encoded as one of the codes 224 .. 448
    assert np.all((q & 0x7F).max(axis=1) >= 0x76)


def test_e4m3_row_scale_edges():
    # a zero row keeps scale 1; a row maximum of exactly 448 * 2^k gives 2^k (not 2^(k+1)); one ulp above
    # gives 2^(k+1); the exponent is clamped to [-126, 127]
    cases = [(0.0, 1.0), (448.0, 1.0), (np.nextafter(np.float32(448.0), np.float32(1e9)), 2.0), (1.0, 2.0 ** -8),
             (1.75, 2.0 ** -8), (np.nextafter(np.float32(1.75), np.float32(9)), 2.0 ** -7), (1e-44, 2.0 ** -126),
             (3e38, 2.0 ** 120)]
    for m, want in cases:
        A = np.array([[1.0, float(np.float32(m))], [0.0, 1.0]])
        _, s = oracle.offdiag_e4m3(A)
        assert s[0] == np.float32(want), (m, s[0], want)
        assert s[1] == 1.0


def test_f32_narrowing_of_edge_values():
    """The FP32 narrow copy rounds FP64 -> FP32 to nearest even (ties, exponent carries, overflow to
    infinity, subnormals, signed zeros), as numpy's conversion does."""
    x = f64_narrowing_cases()
    n = int(np.ceil(np.sqrt(x.size))) + 1
    A = np.eye(n)
    off = ~np.eye(n, dtype=bool)
    A[off] = np.resize(x, off.sum())
    got = oracle.offdiag_f32(A)
    with np.errstate(over="ignore"):
        want = np.where(off, A, 0.0).astype(np.float32)
    np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))


# ---- block-hybrid Gauss-Seidel / SOR --------------------------------------------------------------

def test_block_sor_with_one_block_per_row_is_jacobi():
    """Every row its own block, omega = 1: no in-block predecessor, so each component uses the previous
    iterate only; the iterates equal the Jacobi oracle's bit for bit."""
    A, B, _ = synth.dominant_system(60, 1.15, seed=31, nrhs=2)
    j = oracle.jacobi(A, B, max_iter=300, tol=1e-13, trace=True)
    g = oracle.block_sor(A, B, max_iter=300, tol=1e-13, blocks=60, omega=1.0, trace=True)
    assert (g.status, g.iters) == (j.status, j.iters)
    np.testing.assert_array_equal(g.trace, j.trace)


@pytest.mark.parametrize("blocks", [1, 3])
def test_gauss_seidel_on_block_lower_triangular_is_forward_substitution(blocks):
    """A lower triangular inside each block and zero elsewhere: one Gauss-Seidel sweep is forward
    substitution (scipy's triangular solve gives the same X); the second sweep changes nothing."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(5)
    n = 90
    starts = oracle.uniform_blocks(n, blocks)
    A = np.zeros((n, n))
    for b in range(blocks):
        s0, s1 = starts[b], starts[b + 1]
        L = np.tril(rng.uniform(-1, 1, (s1 - s0, s1 - s0)), -1)
        A[s0:s1, s0:s1] = L + np.diag(rng.uniform(2, 3, s1 - s0) * rng.choice([-1, 1], s1 - s0))
    B = rng.uniform(-1, 1, (n, 1))
    g = oracle.block_sor(A, B, max_iter=10, tol=1e-300, blocks=blocks, trace=True)
    want = np.concatenate([scipy_linalg.solve_triangular(A[s0:s1, s0:s1], B[s0:s1], lower=True)
                           for s0, s1 in zip(starts[:-1], starts[1:])])
    np.testing.assert_allclose(g.trace[0], want, rtol=1e-14, atol=1e-15)
    np.testing.assert_array_equal(g.trace[1], g.trace[0])


def _tridiagonal(n, diag):
    return np.diag(np.full(n, diag)) + np.diag(np.full(n - 1, -1.0), 1) + np.diag(np.full(n - 1, -1.0), -1)


@pytest.mark.parametrize("omega_kind", ["gauss_seidel", "under", "optimal", "over"])
def test_sor_iteration_matrix_matches_young_theory(omega_kind):
    """Classical SOR (one block) on a consistently ordered tridiagonal matrix.  One sweep with B = 0 is
    the linear map x -> M x, so sweeping the unit vectors gives M column by column; its spectral radius
    is Young's: mu^2 for Gauss-Seidel; omega - 1 for omega >= omega_opt = 2 / (1 + sqrt(1 - mu^2));
    ((omega mu + sqrt(omega^2 mu^2 - 4 (omega - 1))) / 2)^2 below it, mu = rho(D^-1 (L + U))."""
    n = 40
    A = _tridiagonal(n, 2.2)
    D = np.diag(np.diag(A))
    mu = max(abs(np.linalg.eigvals(np.eye(n) - np.linalg.solve(D, A))))
    w_opt = 2.0 / (1.0 + np.sqrt(1.0 - mu * mu))
    omega = {"gauss_seidel": 1.0, "under": 0.5 * (1.0 + w_opt), "optimal": w_opt,
             "over": 0.5 * (w_opt + 2.0)}[omega_kind]
    if omega >= w_opt:
        rho = omega - 1.0
    else:
        rho = ((omega * mu + np.sqrt(omega * omega * mu * mu - 4.0 * (omega - 1.0))) / 2.0) ** 2
    g = oracle.block_sor(A, np.zeros((n, n)), X0=np.eye(n), max_iter=1, tol=1e-300, blocks=1, omega=omega,
                         trace=True)
    M = g.trace[0]
    got = max(abs(np.linalg.eigvals(M)))
    # the optimal omega gives a defective eigenvalue: its numerical eigenvalues spread by ~sqrt(eps)
    assert abs(got - rho) <= (2e-7 if omega_kind == "optimal" else 1e-10), (omega_kind, got, rho)


def test_sor_on_a_diagonal_matrix_is_one_relaxed_step():
    """A diagonal: v = b / a_ii is exact, so each sweep moves x by omega (v - x): after k sweeps the error
    is (1 - omega)^k of the start error (closed form)."""
    rng = np.random.default_rng(9)
    n = 25
    d = rng.uniform(1, 2, n) * rng.choice([-1, 1], n)
    A = np.diag(d)
    B = rng.uniform(-1, 1, (n, 1))
    X0 = rng.uniform(-1, 1, (n, 1))
    xs = B / d[:, None]
    for omega in (0.7, 1.0, 1.3):
        g = oracle.block_sor(A, B, X0=X0, max_iter=4, tol=1e-300, blocks=4, omega=omega, trace=True)
        for k in range(len(g.trace)):  # omega = 1 lands on xs in one sweep and stops after the second
            np.testing.assert_allclose(g.trace[k], xs + (1 - omega) ** (k + 1) * (X0 - xs), rtol=0, atol=1e-14)


@pytest.mark.parametrize("blocks,omega", [(1, 1.0), (4, 1.0), (17, 1.0), (1, 1.1), (5, 0.8)])
def test_block_sor_converges_to_the_ge_solution(blocks, omega):
    A, B, Xs = synth.dominant_system(120, 1.2, seed=41, nrhs=2)
    g = oracle.block_sor(A, B, max_iter=500, tol=1e-14, blocks=blocks, omega=omega)
    _, Xge = oracle.ge(A, B)
    assert g.status == 0
    assert np.max(np.abs(g.X - Xge)) <= 1e-12


def test_gauss_seidel_beats_jacobi_on_the_hard_generator():
    """Positive off-diagonals (rho(T) = 1/f): Gauss-Seidel needs a small fraction of Jacobi's sweeps."""
    A, B, _ = synth.hard_system(300, 1.05, seed=3)
    j = oracle.jacobi(A, B, max_iter=5000, tol=1e-10)
    g = oracle.block_sor(A, B, max_iter=5000, tol=1e-10, blocks=1)
    assert j.status == 0 and g.status == 0
    assert g.iters * 10 < j.iters, (g.iters, j.iters)


def test_block_sor_errors():
    A = np.eye(4)
    B = np.ones((4, 1))
    A[1, 1] = 0.0
    assert oracle.block_sor(A, B, blocks=2).status == oracle.ZERO_DIAGONAL
    A[1, 1] = 1.0
    assert oracle.block_sor(A, B, blocks=2, omega=2.0).status == oracle.INVALID_ARG
    assert oracle.block_sor(A, B, blocks=np.array([0, 3, 2, 4])).status == oracle.INVALID_ARG
    assert oracle.block_sor(A, B, blocks=2, norm=oracle.NORM_RESID).status == oracle.INVALID_ARG


# ---- sparse (CSR) Jacobi ------------------------------------------------------------------------------

@pytest.mark.parametrize("norm", [oracle.NORM_INF, oracle.NORM_2, oracle.NORM_RESID])
@pytest.mark.parametrize("kind", ["irregular", "stencil2d"])
def test_csr_jacobi_equals_the_dense_oracle_bit_for_bit(kind, norm):
    """On the dense form of the same matrix the dense oracle adds the zero entries too; adding exact zeros
    leaves an ascending-order FP64 sum unchanged, so every iterate, the sweep count and the final change
    agree bit for bit (rows without off-diagonals and rows 60 entries long included)."""
    if kind == "irregular":
        rp, ci, v, B, _ = synth.random_sparse_system(257, 1.1, seed=21, max_len=60)
    else:
        rp, ci, v, B, _ = synth.stencil_system((13, 11), 1.05, seed=22)
    n = rp.size - 1
    assert kind != "irregular" or np.diff(rp).min() == 1  # some rows hold only the diagonal
    A = synth.csr_to_dense(n, rp, ci, v)
    tol = 1e-11 if norm == oracle.NORM_RESID else 1e-13
    d = oracle.jacobi(A, B, max_iter=400, tol=tol, norm=norm, trace=True)
    s = oracle.csr_jacobi(rp, ci, v, B, max_iter=400, tol=tol, norm=norm, trace=True)
    assert (s.status, s.iters, s.delta) == (d.status, d.iters, d.delta)
    np.testing.assert_array_equal(s.trace, d.trace)
    np.testing.assert_array_equal(s.X, d.X)


@pytest.mark.parametrize("shape,modes", [((23,), (3,)), ((15, 12), (2, 5)), ((7, 9, 6), (1, 4, 2))])
def test_csr_stencil_sine_mode_decays_by_its_eigenvalue(shape, modes):
    """Screened Poisson stencil with unit weights and the constant diagonal a = 2 f dim: T = G / a with G
    the grid's adjacency, whose Dirichlet eigenvectors are products of sines,
    v(i) = prod_d sin(p_d pi (i_d + 1) / (N_d + 1)), eigenvalue sum_d 2 cos(p_d pi / (N_d + 1)).  With
    B = 0 and X0 = v every sweep multiplies by lambda = that / a (closed form)."""
    f = 1.3
    rp, ci, v, _, _ = synth.stencil_system(shape, f, seed=23, weights="unit", diag="constant")
    axes = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    mode = np.ones(shape)
    lam = 0.0
    for ax, N, p in zip(axes, shape, modes):
        mode = mode * np.sin(p * np.pi * (ax + 1) / (N + 1))
        lam += 2.0 * np.cos(p * np.pi / (N + 1))
    lam /= 2.0 * len(shape) * f
    x0 = mode.reshape(-1)
    n = x0.size
    r = oracle.csr_jacobi(rp, ci, v, np.zeros(n), X0=x0, max_iter=6, tol=1e-300, trace=True)
    for k in range(6):
        np.testing.assert_allclose(r.trace[k][:, 0], lam ** (k + 1) * x0, rtol=0, atol=1e-14)


def test_csr_tridiagonal_converges_to_the_direct_solution():
    """1-D variable-coefficient diffusion (tridiagonal): the converged iterate is scipy's banded solve."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rp, ci, v, B, Xs = synth.stencil_system((500,), 1.02, seed=24)
    A = synth.csr_to_dense(500, rp, ci, v)
    ab = np.zeros((3, 500))
    ab[0, 1:] = np.diag(A, 1)
    ab[1] = np.diag(A)
    ab[2, :-1] = np.diag(A, -1)
    want = scipy_linalg.solve_banded((1, 1), ab, B[:, 0])
    r = oracle.csr_jacobi(rp, ci, v, B, max_iter=5000, tol=1e-14)
    assert r.status == oracle.OK
    np.testing.assert_allclose(r.X[:, 0], want, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r.X[:, 0], Xs[:, 0], rtol=0, atol=1e-12)


def test_stencil_generator_structure():
    rp, ci, v, B, Xs = synth.stencil_system((6, 5, 4), 1.05, seed=25)
    n = 120
    A = synth.csr_to_dense(n, rp, ci, v)
    np.testing.assert_array_equal(A, A.T)
    off = A - np.diag(np.diag(A))
    assert np.max(np.abs(off).sum(axis=1) / np.abs(np.diag(A))) == pytest.approx(1 / 1.05, rel=1e-15)
    assert np.diff(rp).max() == 7 and np.diff(rp).min() == 4  # interior 7-point rows, corners 3 + 1
    np.testing.assert_allclose(A @ Xs, B, rtol=0, atol=1e-13)


def test_csr_jacobi_errors():
    rp = np.array([0, 2, 4, 6])
    ci = np.array([0, 1, 0, 1, 1, 2])
    v = np.array([4.0, 1.0, 1.0, 4.0, 1.0, 4.0])
    b = np.ones(3)
    assert oracle.csr_jacobi(rp, ci, v, b).status == oracle.OK
    bad = ci.copy()
    bad[[4, 5]] = [2, 1]  # descending columns
    assert oracle.csr_jacobi(rp, bad, v, b).status == oracle.INVALID_ARG
    bad = ci.copy()
    bad[5] = 1  # repeated column
    assert oracle.csr_jacobi(rp, bad, v, b).status == oracle.INVALID_ARG
    bad = ci.copy()
    bad[5] = 3  # out of range
    assert oracle.csr_jacobi(rp, bad, v, b).status == oracle.INVALID_ARG
    assert oracle.csr_jacobi(np.array([0, 2, 1, 6]), ci, v, b).status == oracle.INVALID_ARG
    missing = np.array([0, 2, 4, 5]), np.array([0, 1, 0, 1, 1]), np.array([4.0, 1.0, 1.0, 4.0, 1.0])
    assert oracle.csr_jacobi(*missing, b).status == oracle.ZERO_DIAGONAL  # row 2 has no diagonal entry
    z = v.copy()
    z[3] = 0.0
    assert oracle.csr_jacobi(rp, ci, z, b).status == oracle.ZERO_DIAGONAL
    z[3] = np.inf
    assert oracle.csr_jacobi(rp, ci, z, b).status == oracle.NONFINITE


def test_csr_residual_equals_the_dense_residual_bit_for_bit():
    """The CSR residual sums the stored entries in column order; the dense one adds exact zeros besides,
    which leaves every FP64 partial sum unchanged: r and the relative residual agree bit for bit."""
    rp, ci, v, B, Xs = synth.random_sparse_system(300, 1.1, seed=26, max_len=50)
    A = synth.csr_to_dense(300, rp, ci, v)
    X = Xs + 1e-3 * np.cos(np.arange(300.0))[:, None]
    Rd, reld = oracle.residual(A, B, X)
    Rs, rels = oracle.csr_residual(rp, ci, v, B, X)
    np.testing.assert_array_equal(Rs, Rd[:, 0])
    assert rels == reld
    _, rel0 = oracle.csr_residual(rp, ci, v, B, Xs)
    assert rel0 <= 1e-15  # the planted solution
