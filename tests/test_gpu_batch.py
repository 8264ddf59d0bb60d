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
    # the whole rollout reversed from step 500 with sqrt(N) checkpoints (the registered states
    # are the initial ones): <lam_500, J v> from the oracle's forward mode over the 500 logged
    # steps equals <lam_0, v> on the two smallest instances
    b.set_states([U.clone() for U in states])
    lam_T = [torch.tensor(rng.standard_normal(U.shape), device="cuda") for U in states]
    lam_0 = [l.clone() for l in lam_T]
    pbs = [torch.zeros(20, dtype=torch.float64, device="cuda") for _ in states]
    b.rollout_vjp(log, lam_0, pbs)
    assert b.status() == 0
    for k in small[:2]:
        p = probs[k]
        U0 = O.prim_to_cons(p, p.W0)
        v = rng.standard_normal(U0.shape) * np.abs(U0).max(axis=(1, 2), keepdims=True) * 1e-3
        _, Jv = O.step_tangent(p, U0, v, np.zeros(20), dts[:, k])
        lam = to_host(lam_T[k])
        lhs = np.dot(lam.reshape(-1), Jv.reshape(-1))
        rhs = np.dot(to_host(lam_0[k]).reshape(-1), v.reshape(-1))
        assert abs(lhs - rhs) <= 1e-10 * np.abs(lam).sum() * np.abs(Jv).max(), (k, lhs, rhs)
    b.close()


# ---------------------------------------------------------------------------------------
# the persistent batched reverse (one launch per reversed step of all instances) and the
# checkpointed rollout reverse
# ---------------------------------------------------------------------------------------
def _mixed_cases():
    """Uneven grids, viscous and Euler instances, immersed bodies of different sizes, and one
    instance without a body (no ghost cells: empty work lists in the IB phases)."""
    out = W.batched_cases(3, seed=21, nx_choices=(64, 96, 128), ny_choices=(48, 64))
    out.append(W.shock_cylinder(nx=80, ny=56, mach=2.4, radius=0.45, viscous=False))
    out.append(W.riemann2d(48, ny=40))
    out.append(W.shock_cylinder(nx=112, ny=40, mach=1.8, radius=0.35, Re=300.0))
    return out


def _per_instance_vjp(torch, B, p, U, dt, lam):
    s = B.Solver.from_problem(p)
    pb = torch.zeros(20, dtype=torch.float64, device="cuda")
    out, _ = s.step_vjp(U, dt, lam, p_bar=pb)
    torch.cuda.synchronize()
    s.close()
    return out, pb


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


def test_persistent_reverse_step_equals_js_step_vjp(env):
    """lambda_n and p_bar of every instance equal js_step_vjp's to rounding (the same device
    bodies on the same elements, inlined into one kernel, where the compiler may fuse a
    different set of products and sums), and a second call reproduces the first bit for bit."""
    torch, B = env
    probs = _mixed_cases()
    states = _states(torch, probs)
    b = B.Batch(probs)
    b.set_states([U.clone() for U in states])
    rng = np.random.default_rng(2)
    lams = [torch.tensor(rng.standard_normal(U.shape), device="cuda") for U in states]
    dts = []
    for p, U in zip(probs, states):
        s = B.Solver.from_problem(p)
        dts.append(0.9 * s.max_dt(U, 0.5))
        s.close()
    outs = [torch.empty_like(U) for U in states]
    pbs = [torch.zeros(20, dtype=torch.float64, device="cuda") for _ in states]
    b.step_vjp(states, dts, lams, outs, pbs)
    assert b.status() == 0
    for k, p in enumerate(probs):
        ref, pref = _per_instance_vjp(torch, B, p, states[k], dts[k], lams[k])
        print("instance %d: lambda %.2e, p_bar %.2e (relative to the maxima)" % (k, _rel(outs[k], ref),
                                                                             _rel(pbs[k], pref)))
        assert _rel(outs[k], ref) < 1e-13, k
        assert _rel(pbs[k], pref) < 1e-12, k
    # lam_n may alias lam_np1; the same call again gives the same bits
    again = [lam.clone() for lam in lams]
    pb2 = [torch.zeros(20, dtype=torch.float64, device="cuda") for _ in states]
    b.step_vjp(states, dts, again, again, pb2)
    assert b.status() == 0
    for k in range(len(probs)):
        assert torch.equal(again[k], outs[k]), k
        assert torch.equal(pb2[k], pbs[k]), k
    b.close()


def test_split_reverse_launch_equals_the_persistent_launch(env):
    """One launch per phase (js_batch_set_reverse_launch(b, 1)) runs the persistent kernel's
    device code on the same work items in the same order: lambda_n and p_bar equal the
    persistent launch's to rounding (separately compiled kernels may contract a different set of
    products into fused multiply-adds) and repeat bit for bit; a rollout reverse with the split
    launch (stage states given) equals the per-instance step-by-step reverse."""
    torch, B = env
    probs = _mixed_cases()
    states = _states(torch, probs)
    b = B.Batch(probs)
    b.set_states([U.clone() for U in states])
    assert b.reverse_launch() == 0
    with pytest.raises(B.JsError):
        b.set_reverse_launch(2)
    rng = np.random.default_rng(12)
    lams = [torch.tensor(rng.standard_normal(U.shape), device="cuda") for U in states]
    dts = []
    for p, U in zip(probs, states):
        s = B.Solver.from_problem(p)
        dts.append(0.9 * s.max_dt(U, 0.5))
        s.close()
    res = {}
    for split in (0, 1, 1):
        b.set_reverse_launch(split)
        assert b.reverse_launch() == split
        outs = [torch.empty_like(U) for U in states]
        pbs = [torch.zeros(20, dtype=torch.float64, device="cuda") for _ in states]
        b.step_vjp(states, dts, lams, outs, pbs)
        assert b.status() == 0
        if split in res:  # the second split call: the same bits
            for k in range(len(probs)):
                assert torch.equal(outs[k], res[split][0][k]), k
                assert torch.equal(pbs[k], res[split][1][k]), k
        res[split] = (outs, pbs)
    for k in range(len(probs)):
        assert _rel(res[1][0][k], res[0][0][k]) < 1e-13, k
        assert _rel(res[1][1][k], res[0][1][k]) < 1e-12, k
    # rollout reverse (stage states given to the reverse launches) with the split launch
    n = 7
    log = torch.zeros((n, len(probs)), dtype=torch.float64, device="cuda")
    for k, (p, U) in enumerate(zip(probs, states)):
        log[:, k] = torch.tensor(dts[k] * rng.uniform(0.5, 0.9, n))
    work = [lam.clone() for lam in lams]
    pbs = [torch.zeros(20, dtype=torch.float64, device="cuda") for _ in states]
    b.rollout_vjp(log, work, pbs, ckpt=3)
    assert b.status() == 0
    for k, p in enumerate(probs):
        ref, pref = _reference_rollout_reverse(torch, B, p, states[k], log[:, k].tolist(), lams[k])
        assert _rel(work[k], ref) < 1e-12, (k, _rel(work[k], ref))
        assert _rel(pbs[k], pref) < 1e-11, (k, _rel(pbs[k], pref))
    b.close()


def test_fixed_step_sizes_replay_per_instance_steps(env):
    torch, B = env
    probs = _mixed_cases()
    states = _states(torch, probs)
    b = B.Batch(probs)
    work = [U.clone() for U in states]
    b.set_states(work)
    rng = np.random.default_rng(4)
    dts = torch.zeros((6, len(probs)), dtype=torch.float64, device="cuda")
    for k, (p, U) in enumerate(zip(probs, states)):
        s = B.Solver.from_problem(p)
        dts[:, k] = torch.tensor(s.max_dt(U, 0.5) * rng.uniform(0.5, 0.9, 6))
        s.close()
    b.step_fixed(dts)
    assert b.status() == 0
    for k, (p, U) in enumerate(zip(probs, states)):
        s = B.Solver.from_problem(p)
        V = U.clone()
        for j in range(6):
            s.step(V, float(dts[j, k]), 1)
        assert torch.equal(V, work[k]), k
        s.close()
    b.close()


def _reference_rollout_reverse(torch, B, p, U0, dts, lam):
    """Per instance: the forward states by js_step, then js_step_vjp from the last step back."""
    s = B.Solver.from_problem(p)
    states = [U0.clone()]
    for dt in dts:
        V = states[-1].clone()
        s.step(V, dt, 1)
        states.append(V)
    lam = lam.clone()
    pb = torch.zeros(20, dtype=torch.float64, device="cuda")
    for j in range(len(dts) - 1, -1, -1):
        s.step_vjp(states[j], dts[j], lam, lam_n=lam, p_bar=pb)
    torch.cuda.synchronize()
    s.close()
    return lam, pb


@pytest.mark.parametrize("ckpt", [4, 0, 13])
def test_rollout_reverse_equals_step_by_step_reverse(env, ckpt):
    """13 steps, checkpoints every ckpt (4: an uneven last segment; 0: the library's choice,
    every state for a batch this small; 13: one segment): dL/dU_0 equals the per-instance
    step-by-step reverse to rounding, and the same for every checkpoint spacing bit for bit;
    the registered states are left unchanged."""
    torch, B = env
    probs = _mixed_cases()
    states = _states(torch, probs)
    b = B.Batch(probs)
    reg = [U.clone() for U in states]
    b.set_states(reg)
    n = 13
    rng = np.random.default_rng(6)
    dts = torch.zeros((n, len(probs)), dtype=torch.float64, device="cuda")
    for k, (p, U) in enumerate(zip(probs, states)):
        s = B.Solver.from_problem(p)
        dts[:, k] = torch.tensor(s.max_dt(U, 0.5) * rng.uniform(0.4, 0.8, n))
        s.close()
    lams = [torch.tensor(rng.standard_normal(U.shape), device="cuda") for U in states]
    work = [lam.clone() for lam in lams]
    pbs = [torch.zeros(20, dtype=torch.float64, device="cuda") for _ in states]
    b.rollout_vjp(dts, work, pbs, ckpt=ckpt)
    assert b.status() == 0
    for k, p in enumerate(probs):
        assert torch.equal(reg[k], states[k]), k
        ref, pref = _reference_rollout_reverse(torch, B, p, states[k], dts[:, k].tolist(), lams[k])
        assert _rel(work[k], ref) < 1e-12, (k, _rel(work[k], ref))
        assert _rel(pbs[k], pref) < 1e-11, (k, _rel(pbs[k], pref))
    # another checkpoint spacing: the same segments' states, the same reverse launches
    other = [lam.clone() for lam in lams]
    b.rollout_vjp(dts, other, None, ckpt=1 if ckpt != 1 else 2)
    assert b.status() == 0
    for k in range(len(probs)):
        assert torch.equal(other[k], work[k]), k
    b.close()


def test_rollout_default_spacing(env):
    """With ckpt = 0 the rollout keeps every state when they fit in half the free memory (this
    batch's 15 states do), and reuses the spacing of a workspace already prepared for the same
    step count; the square-root spacing otherwise."""
    torch, B = env
    probs = _mixed_cases()
    states = _states(torch, probs)
    b = B.Batch(probs)
    b.set_states([U.clone() for U in states])
    assert b.rollout_spacing(13) == 1
    dts = torch.zeros((13, len(probs)), dtype=torch.float64, device="cuda")
    b.rollout_forward(0.5, dts, ckpt=4)
    assert b.rollout_spacing(13) == 4 and b.rollout_spacing(12) == 1
    b.close()


@pytest.mark.parametrize("split", [0, 1])
def test_rollout_reverse_is_graph_capturable(env, split):
    torch, B = env
    probs = _mixed_cases()[:3]
    states = _states(torch, probs)
    side = torch.cuda.Stream()
    n = 9
    with torch.cuda.stream(side):
        b = B.Batch(probs, stream=side)
        b.set_reverse_launch(split)
        b.set_states([U.clone() for U in states])
        log = torch.zeros((n, len(probs)), dtype=torch.float64, device="cuda")
        fwd = [U.clone() for U in states]
        b.set_states(fwd)
        b.step(0.5, n, dt_log=log)
        b.set_states([U.clone() for U in states])
        rng = np.random.default_rng(8)
        lam0 = [torch.tensor(rng.standard_normal(U.shape), device="cuda") for U in states]
        eager = [l.clone() for l in lam0]
        b.rollout_vjp(log, eager, ckpt=3)  # first call: workspace, tables
        work = [l.clone() for l in lam0]
        b.rollout_vjp(log, work, ckpt=3)  # same pointers from here on
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            b.rollout_vjp(log, work, ckpt=3)
    torch.cuda.synchronize()
    for w, l in zip(work, lam0):
        w.copy_(l)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert b.status() == 0
    for w, e in zip(work, eager):
        assert torch.equal(w, e)
    b.close()


def test_launch_tuning_keeps_results_and_the_tuner_caches_its_choice(env, tmp_path, monkeypatch):
    """Every (blocks per SM, schedule) gives the default launch's states bit for bit; the
    autotuner times them, applies the fastest and finds it in its cache the next time."""
    torch, B = env
    from paper_2601_04400_gb300 import tuning
    monkeypatch.setattr(tuning, "_CACHE", str(tmp_path / "tuning.json"))
    probs = _mixed_cases()
    states = _states(torch, probs)
    b = B.Batch(probs)
    ref = [U.clone() for U in states]
    b.set_states(ref)
    b.step(0.5, 3)
    _, most, _, nsched = b.tuning()
    assert most >= 1 and nsched == 3
    for bps in range(1, most + 1):
        for sched in range(nsched):
            b.set_tuning(bps, sched)
            assert b.tuning()[0] == bps and b.tuning()[2] == sched
            work = [U.clone() for U in states]
            b.set_states(work)
            b.step(0.5, 3)
            assert b.status() == 0
            for w, r in zip(work, ref):
                assert torch.equal(w, r), (bps, sched)
    times = tuning.autotune_batch(b, probs, states)
    assert len(times) == most * nsched
    choice = b.tuning()
    b.set_tuning(0, 0)
    assert tuning.autotune_batch(b, probs, states) == {}
    assert b.tuning() == choice
    b.close()


def test_rollout_forward_keeps_checkpoints_for_the_reverse(env):
    """js_batch_rollout_forward = js_batch_step with the CFL rule (states and logged step sizes bit
    for bit); the reverse that follows reuses its checkpoints and equals a reverse that runs its
    own forward from the initial states."""
    torch, B = env
    probs = _mixed_cases()
    states = _states(torch, probs)
    n = 11
    b = B.Batch(probs)
    plain = [U.clone() for U in states]
    b.set_states(plain)
    log_a = torch.zeros((n, len(probs)), dtype=torch.float64, device="cuda")
    b.step(0.5, n, dt_log=log_a)
    fwd = [U.clone() for U in states]
    b.set_states(fwd)
    log_b = torch.zeros((n, len(probs)), dtype=torch.float64, device="cuda")
    b.rollout_forward(0.5, log_b, ckpt=3)
    assert b.status() == 0
    assert torch.equal(log_a, log_b)
    for x, y in zip(fwd, plain):
        assert torch.equal(x, y)
    rng = np.random.default_rng(12)
    lam_T = [torch.tensor(rng.standard_normal(U.shape), device="cuda") for U in states]
    reuse = [l.clone() for l in lam_T]
    b.rollout_vjp(log_b, reuse, ckpt=3)
    b.set_states([U.clone() for U in states])
    fresh = [l.clone() for l in lam_T]
    b.rollout_vjp(log_b, fresh, ckpt=3)
    assert b.status() == 0
    for x, y in zip(reuse, fresh):
        assert torch.equal(x, y)
    b.close()
