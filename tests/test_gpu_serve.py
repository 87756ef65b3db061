"""Serving (continuous batching) on the GPU.

* The device generator reproduces synth.serving_request bit for bit (integer work: exact equality).
* Every served request meets ||B - A X||_inf / ||B||_inf <= 1e-10 per column, recomputed by the oracle in
  FP64 on inputs regenerated on the host.
* A request's result is identical alone and in a mix of other requests admitted at different rounds.
* Admission respects the memory budget: with room for a few requests, the rest wait and all finish.
* A request with a zero diagonal fails alone; an oversized request is refused at submission.
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


@pytest.mark.parametrize("n,r,f,seed", [(1, 1, 1.2, 3), (7, 3, 1.05, 11), (300, 16, 1.3, 12345), (1025, 5, 1.5, 99)])
def test_device_generator_is_bit_exact(jac, n, r, f, seed):
    A, B = jac.generate_request(n, r, f, seed)
    Ah, Bh = synth.serving_request(n, r, f, seed)
    np.testing.assert_array_equal(A.cpu().numpy(), Ah)
    np.testing.assert_array_equal(B.cpu().numpy().T, Bh)


def drain(srv, limit=100000):
    done = {}
    for _ in range(limit):
        a, p = srv.step()
        for rid, st in srv.poll():
            done[rid] = st
        if a == 0 and p == 0:
            break
    for rid, st in srv.poll():
        done[rid] = st
    return done


RESIDUALS = ["fp64", "split", "tc"]


def make_server(jac, budget, residual, **kw):
    return jac.Server(budget_bytes=budget, split_residual=residual == "split", tc_residual=residual == "tc", **kw)


@pytest.mark.parametrize("residual", RESIDUALS)
def test_served_requests_reach_target(jac, residual):
    """The residual rounds by FP64 FMAs, by the split-float arithmetic (FP32 units), or on the tensor cores
    from the digit split of A and X."""
    import torch
    t, ns, rs, fs, seeds = synth.serving_trace(2000, 0.02, seed=4, n_lo=64, n_hi=1500)
    srv = make_server(jac, 2 << 30, residual)
    outs, ids = {}, {}
    for k in range(len(t)):
        out = torch.full((int(rs[k]), int(ns[k])), float("nan"), dtype=torch.float64, device="cuda")
        rid = srv.submit_generated(int(ns[k]), int(rs[k]), float(fs[k]), int(seeds[k]), out)
        ids[rid] = k
        outs[rid] = out
    done = drain(srv)
    assert set(done) == set(ids)
    for rid, st in done.items():
        k = ids[rid]
        A, B = synth.serving_request(int(ns[k]), int(rs[k]), float(fs[k]), int(seeds[k]))
        X = outs[rid].cpu().numpy().T
        _, rel = oracle.residual(A, B, X)
        assert st.status == 0 and rel <= 1e-10, (k, ns[k], rs[k], st.as_dict(), rel)
        assert abs(st.rel_residual - rel) <= (5e-13 if residual == "split" else 1e-13) + 1e-3 * rel


@pytest.mark.parametrize("residual", RESIDUALS)
def test_result_is_the_same_alone_and_in_the_mix(jac, residual):
    import torch
    probe = (700, 4, 1.1, 777)
    alone = make_server(jac, 1 << 30, residual)
    xa = torch.zeros(4, 700, dtype=torch.float64, device="cuda")
    alone.submit_generated(*probe, xa)
    drain(alone)
    mix = make_server(jac, 1 << 30, residual)
    xm = torch.zeros(4, 700, dtype=torch.float64, device="cuda")
    others = []
    for k, (n, r) in enumerate([(1200, 16), (64, 1), (333, 7)]):
        o = torch.zeros(r, n, dtype=torch.float64, device="cuda")
        mix.submit_generated(n, r, 1.2, 1000 + k, o)
        others.append(o)
    mix.step()
    mix.step()  # the probe arrives while the others are already on the device
    mix.submit_generated(*probe, xm)
    for k, (n, r) in enumerate([(2000, 2), (90, 9)]):
        o = torch.zeros(r, n, dtype=torch.float64, device="cuda")
        mix.submit_generated(n, r, 1.3, 2000 + k, o)
        others.append(o)
    drain(mix)
    assert torch.equal(xa, xm)


def test_admission_respects_the_budget(jac):
    import torch
    n, r = 1000, 8
    per_request = 1000 * 1000 * 8 + 1000 * 1008 * 4 + 6 * 8 * 1008 * 8  # A + FP32 copy + vectors (approx.)
    srv = jac.Server(budget_bytes=int(2.5 * per_request))
    outs = [torch.zeros(r, n, dtype=torch.float64, device="cuda") for _ in range(6)]
    for k in range(6):
        srv.submit_generated(n, r, 1.2, 50 + k, outs[k])
    a, p = srv.step()
    assert a == 2 and p == 4  # only two fit at a time
    done = drain(srv)
    assert len(done) == 6 and all(st.status == 0 for st in done.values())


def test_bad_request_and_oversized_request(jac):
    import torch
    srv = jac.Server(budget_bytes=256 << 20)
    A = torch.eye(5, dtype=torch.float64, device="cuda")
    A[2, 2] = 0.0
    B = torch.ones(1, 5, dtype=torch.float64, device="cuda")
    xbad = torch.zeros(1, 5, dtype=torch.float64, device="cuda")
    rb = srv.submit(A, B, xbad)
    xok = torch.zeros(2, 200, dtype=torch.float64, device="cuda")
    rk = srv.submit_generated(200, 2, 1.2, 5, xok)
    done = drain(srv)
    assert done[rb].status == jac.ERR_ZERO_DIAGONAL
    assert done[rk].status == 0
    with pytest.raises(jac.JacobiError) as e:
        srv.submit_generated(8192, 16, 1.2, 6, torch.zeros(16, 8192, dtype=torch.float64, device="cuda"))
    assert e.value.status == jac.ERR_OUT_OF_MEMORY


def test_wait_for_one_request(jac):
    """jacobi_server_wait runs rounds until the named request is done and collects it; requests that finish
    meanwhile stay for poll; an unknown or collected id is rejected."""
    import torch
    srv = jac.Server(budget_bytes=1 << 30)
    outs, ids = [], []
    for k, (n, r) in enumerate([(900, 3), (120, 1), (2500, 8), (64, 2)]):
        o = torch.zeros(r, n, dtype=torch.float64, device="cuda")
        ids.append(srv.submit_generated(n, r, 1.2, 500 + k, o))
        outs.append(o)
    st = srv.wait(ids[2])
    A, B = synth.serving_request(2500, 8, 1.2, 502)
    _, rel = oracle.residual(A, B, outs[2].cpu().numpy().T)
    assert st.status == 0 and rel <= 1e-10
    with pytest.raises(jac.JacobiError) as e:
        srv.wait(ids[2])
    assert e.value.status == jac.ERR_INVALID_ARG
    rest = drain(srv)
    assert set(rest) == {ids[0], ids[1], ids[3]}
    with pytest.raises(jac.JacobiError):
        srv.wait(12345)


@pytest.mark.parametrize("residual", RESIDUALS)
def test_zero_right_hand_side_columns(jac, residual):
    """The server's reading of a zero right-hand side: a zero column of B is solved exactly by its zero
    start and counts as met.  A request with B = 0 finishes OK with X = 0; in a request whose second column
    is zero that column stays 0 and the others meet 1e-10 by the oracle."""
    import torch
    srv = make_server(jac, 1 << 30, residual)
    A0, _, _ = synth.dominant_system(200, 1.3, seed=81, nrhs=2)
    A1, B1, _ = synth.dominant_system(300, 1.3, seed=82, nrhs=3)
    B1[:, 1] = 0.0
    x0 = torch.ones(2, 200, dtype=torch.float64, device="cuda")
    x1 = torch.ones(3, 300, dtype=torch.float64, device="cuda")
    r0 = srv.submit(torch.from_numpy(A0).cuda(), torch.zeros(2, 200, dtype=torch.float64, device="cuda"), x0)
    r1 = srv.submit(torch.from_numpy(A1).cuda(), torch.from_numpy(np.ascontiguousarray(B1.T)).cuda(), x1)
    done = drain(srv)
    assert done[r0].status == 0 and int(torch.count_nonzero(x0)) == 0
    X1 = x1.cpu().numpy().T
    assert done[r1].status == 0 and not X1[:, 1].any()
    for c in (0, 2):
        _, rel = oracle.residual(A1, B1[:, c:c + 1], X1[:, c:c + 1])
        assert rel <= 1e-10, (c, rel)


def test_tc_residual_rounds_wild_scales(jac):
    """Requests whose A rows and B columns span 2^-60 .. 2^60 (inside the range of the FP32 copy the inner
    sweeps read): the tensor-core residual rounds scale each row and column by its own power of two, so every
    request still meets 1e-10 by the oracle."""
    import torch
    rng = np.random.default_rng(8)
    srv = make_server(jac, 1 << 30, "tc")
    cases = []
    for k, (n, r) in enumerate([(257, 3), (640, 16), (100, 1)]):
        A, B, _ = synth.dominant_system(n, 1.2, seed=70 + k, nrhs=r)
        rows = 2.0 ** rng.integers(-60, 60, n)
        cols = 2.0 ** rng.integers(-60, 60, r)
        A = A * rows[:, None]
        B = B * rows[:, None] * cols[None, :]
        out = torch.zeros(r, n, dtype=torch.float64, device="cuda")
        rid = srv.submit(torch.from_numpy(A).cuda(), torch.from_numpy(np.ascontiguousarray(B.T)).cuda(), out)
        cases.append((rid, A, B, out))
    done = drain(srv)
    for rid, A, B, out in cases:
        _, rel = oracle.residual(A, B, out.cpu().numpy().T)
        assert done[rid].status == 0 and rel <= 1e-10, (done[rid].as_dict(), rel)
