"""The batched persistent path (js_batch_*): many shock-cylinder instances with seeded Mach
numbers, radii and uneven grids, advanced in one launch with per-instance device CFL steps.
It must equal per-instance js_max_dt + js_step runs bit for bit, match the oracle, be
capturable in a CUDA graph, and report a barrier that cannot complete as JS_ERR_TIMEOUT
without hanging."""
import numpy as np
import pytest

import oracle as O
from paper_2601_04400_gb300 import workloads as W
from jsutil import TOL, normwise_err, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04400_gb300 import binding as B
    B.lib()
    return torch, B


def _cases(count=5, seed=3):
    return W.batched_cases(count, seed=seed, nx_choices=(64, 96, 128), ny_choices=(48, 64))


def _states(torch, problems):
    return [torch.tensor(O.prim_to_cons(p, p.W0), device="cuda") for p in problems]


def _sequential(torch, B, problems, states, cfl, n):
    out, times = [], []
    for p, U in zip(problems, states):
        s = B.Solver.from_problem(p)
        U = U.clone()
        t = 0.0
        for _ in range(n):
            dt = s.max_dt(U, cfl)
            s.step(U, dt, 1)
            t += dt
        out.append(to_host(U))
        times.append(t)
        s.close()
    return out, times


def test_batch_equals_per_instance_steps_bitwise(env):
    torch, B = env
    probs = _cases()
    states = _states(torch, probs)
    ref, ref_t = _sequential(torch, B, probs, states, 0.5, 8)
    b = B.Batch(probs)
    work = [U.clone() for U in states]
    b.set_states(work)
    t = torch.zeros(len(probs), dtype=torch.float64, device="cuda")
    b.step(0.5, 5, t)
    b.step(0.5, 3, t)
    assert b.status() == 0
    for k, U in enumerate(work):
        assert np.array_equal(to_host(U), ref[k]), k
    assert np.array_equal(to_host(t), np.array(ref_t))
    b.close()


def test_batch_matches_oracle(env):
    torch, B = env
    probs = _cases(2, seed=5)
    states = _states(torch, probs)
    b = B.Batch(probs)
    work = [U.clone() for U in states]
    b.set_states(work)
    b.step(0.5, 4)
    assert b.status() == 0
    for p, U in zip(probs, work):
        Uo = O.prim_to_cons(p, p.W0)
        for _ in range(4):
            Uo = O.step(p, Uo, [O.max_dt(p, Uo, 0.5)])
        assert normwise_err(to_host(U), Uo) < TOL


def test_batch_step_is_graph_capturable(env):
    torch, B = env
    probs = _cases(3, seed=7)
    states = _states(torch, probs)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        b = B.Batch(probs, stream=side)
        eager = [U.clone() for U in states]
        b.set_states(eager)
        b.step(0.5, 4)
        torch.cuda.synchronize()
        work = [U.clone() for U in states]
        b.set_states(work)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            b.step(0.5, 2)
    torch.cuda.synchronize()
    for U, U0 in zip(work, states):
        U.copy_(U0)
    torch.cuda.synchronize()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert b.status() == 0
    for a, e in zip(work, eager):
        assert np.array_equal(to_host(a), to_host(e))


def test_barrier_timeout_is_reported_and_recoverable(env):
    torch, B = env
    probs = _cases(2, seed=9)
    states = _states(torch, probs)
    b = B.Batch(probs)
    work = [U.clone() for U in states]
    b.set_states(work)
    b.test_timeout(0.05)
    assert b.status() == B.JS_ERR_TIMEOUT
    # the context stays usable: a normal launch afterwards is correct
    for U, U0 in zip(work, states):
        U.copy_(U0)
    b.step(0.5, 2)
    assert b.status() == 0
    ref, _ = _sequential(torch, B, probs, states, 0.5, 2)
    for k, U in enumerate(work):
        assert np.array_equal(to_host(U), ref[k])


def test_batched_reverse_step_matches_oracle_tangent(env):
    """One batched step with logged device dt, then js_batch_step_vjp: <lam, J v> from the
    oracle's forward mode equals <J^T lam, v> for every instance."""
    torch, B = env
    probs = _cases(3, seed=11)
    states = _states(torch, probs)
    b = B.Batch(probs)
    work = [U.clone() for U in states]
    b.set_states(work)
    log = torch.zeros((1, len(probs)), dtype=torch.float64, device="cuda")
    b.step(0.5, 1, dt_log=log)
    assert b.status() == 0
    dts = to_host(log)[0].tolist()
    rng = np.random.default_rng(5)
    lams = [torch.tensor(rng.standard_normal(U.shape), device="cuda") for U in states]
    outs = [torch.empty_like(U) for U in states]
    pbs = [torch.zeros(20, dtype=torch.float64, device="cuda") for _ in states]
    b.step_vjp(states, dts, lams, outs, pbs)
    assert b.status() == 0
    for p, U, lam, Ub, dt in zip(probs, states, lams, outs, dts):
        U0 = to_host(U)
        assert dt == O.max_dt(p, U0, 0.5)
        v = rng.standard_normal(U0.shape) * np.abs(U0).max(axis=(1, 2), keepdims=True) * 1e-3
        _, Jv = O.step_tangent(p, U0, v, np.zeros(20), [dt])
        lhs = np.dot(to_host(lam).reshape(-1), Jv.reshape(-1))
        rhs = np.dot(to_host(Ub).reshape(-1), v.reshape(-1))
        assert abs(lhs - rhs) <= 1e-12 * np.abs(to_host(lam)).sum() * np.abs(Jv).max()


def test_full_batched_configuration(env):
    """The batched configuration itself: the 256 seeded instances (Mach U[1.5,3], radius U[0.3,0.7],
    nx 128..512, ny 128..256, seed 0), 500 steps in ONE launch with per-instance device CFL steps
    (logged).  The three smallest instances, advanced by the oracle with its own CFL steps, agree
    within the 1e-10 bar and their step sequences to rounding; a sample of others, re-run one at a
    time with js_max_dt + js_step, reproduce every logged step and the final state bit for bit; one
    batched reverse step of all 256 instances passes the dot-product test against the oracle's
    forward mode on the three smallest."""
    torch, B = env
    n_steps = 500
    probs = W.batched_cases(256, seed=0)
    states = _states(torch, probs)
    b = B.Batch(probs)
    work = [U.clone() for U in states]
    b.set_states(work)
    log = torch.zeros((n_steps, len(probs)), dtype=torch.float64, device="cuda")
    b.step(0.5, n_steps, dt_log=log)
    assert b.status() == 0
    dts = to_host(log)
    cells = [p.nx * p.ny for p in probs]
    order = sorted(range(len(probs)), key=lambda k: (cells[k], k))
    small = order[:3]
    for k in small:
        p = probs[k]
        Uo = O.prim_to_cons(p, p.W0)
        seq = []
        for _ in range(n_steps):
            dt = O.max_dt(p, Uo, 0.5)
            seq.append(dt)
            Uo = O.step(p, Uo, [dt])
        assert np.abs(np.array(seq) - dts[:, k]).max() <= 1e-12 * dts[:, k].max(), k
        assert normwise_err(to_host(work[k]), Uo) < TOL, k
    for k in (order[len(order) // 2], order[-1], 0, 255):
        p = probs[k]
        s = B.Solver.from_problem(p)
        U = states[k].clone()
        for j in range(n_steps):
            dt = s.max_dt(U, 0.5)
            assert dt == dts[j, k], (k, j)
            s.step(U, dt, 1)
        assert torch.equal(U, work[k]), k
        s.close()
    # one batched reverse step from the initial states (their first logged steps are the
    # oracle's own CFL steps)
    rng = np.random.default_rng(13)
    lams = [torch.tensor(rng.standard_normal(U.shape), device="cuda") for U in states]
    outs = [torch.empty_like(U) for U in states]
    pbs = [torch.zeros(20, dtype=torch.float64, device="cuda") for _ in states]
    b.step_vjp(states, dts[0].tolist(), lams, outs, pbs)
    assert b.status() == 0
    for k in small:
        p = probs[k]
        U0 = O.prim_to_cons(p, p.W0)
        dt = O.max_dt(p, U0, 0.5)
        assert dt == dts[0, k]
        v = rng.standard_normal(U0.shape) * np.abs(U0).max(axis=(1, 2), keepdims=True) * 1e-3
        _, Jv = O.step_tangent(p, U0, v, np.zeros(20), [dt])
        lam = to_host(lams[k])
        lhs = np.dot(lam.reshape(-1), Jv.reshape(-1))
        rhs = np.dot(to_host(outs[k]).reshape(-1), v.reshape(-1))
        assert abs(lhs - rhs) <= 1e-12 * np.abs(lam).sum() * np.abs(Jv).max(), k
    b.close()
