"""Stage-wise entry points and the single-grid y-slab decomposition through the CUDA path.

* js_step_stage x3 equals js_step bitwise; js_step_stage_vjp (2, 1, 0) equals js_step_vjp
  (to 1e-13 relative: the reverse of the first two stages recomputes WENO internals that
  js_step_vjp keeps) and rejects any other order.
* Slabs of one grid held by one process (LocalTransport, one GPU, separate contexts run one
  after another; no kernel waits on another): the owned rows after several steps are
  bitwise equal to the undecomposed grid (every owned cell sees the same inputs and the same
  arithmetic), the CFL steps are equal, and the reverse step equals js_step_vjp on the owned
  rows and in the parameter gradient (summed over slabs: 1e-12 relative).  Cases: the
  four-quadrant problem (transmissive), a periodic viscous grid with artificial viscosity
  (windows that wrap), and a viscous shock-cylinder whose immersed body is cut by the slab
  boundaries (inflow and reflective sides; overlap deep enough for the image points).
* js_create_slab refuses an overlap too shallow for the body's image points (JS_ERR_IB).
* Two processes, one slab each, exchanging through torch.distributed (gloo, host copies) on
  the same GPU: equal to the undecomposed grid."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2601_04400_gb300 import parallel
from paper_2601_04400_gb300 import workloads as W
from jsutil import normwise_err, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04400_gb300 import binding as B
    B.lib()
    return torch, B


def _cylinder():
    p = W.shock_cylinder(nx=70, ny=45, Lx=3.5, Ly=2.25, centre=(1.6, 1.1), radius=0.45, x_shock=0.8, viscous=True)
    return p, O.prim_to_cons(p, W.random_state(p, seed=2, amp=0.02))


def _cases():
    p = W.riemann2d(96, ny=90)
    yield "riemann2d_96x90", p, O.prim_to_cons(p, p.W0), 3
    p = W.random_periodic(64, 60, seed=1, mu=3e-3, nu=1e-3)
    yield "ns_av_periodic_64x60", p, O.prim_to_cons(p, p.W0), 4
    p, U = _cylinder()
    yield "ns_cylinder_ib_70x45", p, U, 14


CASES = list(_cases())


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_stage_entry_points_equal_step_and_step_vjp(env, case):
    torch, B = env
    _, prob, U, _ = case
    s = B.Solver.from_problem(prob)
    Ud = to_dev(U)
    dt = 0.8 * s.max_dt(Ud, 0.5)
    ref = s.step(Ud.clone(), dt, 1)
    X1 = s.step_stage(None, Ud, torch.empty_like(Ud), dt, 0)
    X2 = s.step_stage(Ud, X1, torch.empty_like(Ud), dt, 1)
    out = s.step_stage(Ud, X2, X2, dt, 2)  # output aliasing its input
    assert torch.equal(out, ref)
    lam = to_dev(np.random.default_rng(3).standard_normal(U.shape))
    l_ref, p_ref = s.step_vjp(Ud, dt, lam)
    p = torch.zeros_like(p_ref)
    L = lam.clone()
    X2s = s.step_stage(Ud, X1, torch.empty_like(Ud), dt, 1)  # X2 was overwritten by stage 2
    for k, X in ((2, X2s), (1, X1), (0, Ud)):
        s.step_stage_vjp(X, dt, k, L, L, p)
    assert float((L - l_ref).abs().max()) <= 1e-13 * float(l_ref.abs().max())
    assert float((p - p_ref).abs().max()) <= 1e-13 * float(p_ref.abs().max())
    with pytest.raises(B.JsError):
        s.step_stage_vjp(X2s, dt, 1, L, L, p)  # a step's reverse starts with stage 2
    s.step_stage_vjp(X2s, dt, 2, L, L, p)
    with pytest.raises(B.JsError):
        s.step_stage_vjp(Ud, dt, 0, L, L, p)
    # stages 0 and 1 storing their WENO5 internals, their reverse using them: the same result
    if prob.ny > 1:
        s.step_vjp(Ud, dt, lam)  # reuses the internals' workspace: none are stored now
        L2 = lam.clone()
        s.step_stage_vjp(X2s, dt, 2, L2, L2, None)
        with pytest.raises(B.JsError):
            s.step_stage_vjp(X1, dt, 1, L2, L2, None, internals=True)
        X1k = s.step_stage(None, Ud, torch.empty_like(Ud), dt, 0, internals=True)
        X2k = s.step_stage(Ud, X1k, torch.empty_like(Ud), dt, 1, internals=True)
        assert torch.equal(X1k, X1) and torch.equal(X2k, X2s)
        p2 = torch.zeros_like(p_ref)
        L2 = lam.clone()
        for k, X in ((2, X2k), (1, X1k), (0, Ud)):
            s.step_stage_vjp(X, dt, k, L2, L2, p2, internals=k < 2)
        assert float((L2 - l_ref).abs().max()) <= 1e-13 * float(l_ref.abs().max())
        assert float((p2 - p_ref).abs().max()) <= 1e-13 * float(p_ref.abs().max())
    assert s.status() == 0


def _group(B, prob, world, ov):
    plan = parallel.SlabPlan(prob.ny, world, ov, periodic=prob.bc[2] == 2)
    return parallel.SlabGroup.build(prob, plan, range(world))


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_slabs_forward_equal_whole_grid(env, case, world):
    torch, B = env
    _, prob, U, ov = case
    s = B.Solver.from_problem(prob)
    G = _group(B, prob, world, ov)
    Ud = to_dev(U)
    X = G.scatter(Ud)
    dts = []
    for _ in range(6):
        dt = s.max_dt(Ud, 0.5)
        assert G.max_dt(X, 0.5) == dt
        dts.append(dt)
        s.step(Ud, dt, 1)
        G.step(X, dt, 1)
    out = G.gather(X)
    assert torch.equal(out, Ud), float((out - Ud).abs().max())
    assert normwise_err(to_host(out), O.step(prob, U, dts)) < 1e-10
    for r, sl in G.slabs.items():
        assert sl.status() == 0


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_slabs_reverse_equal_whole_grid(env, case, world):
    torch, B = env
    _, prob, U, ov = case
    s = B.Solver.from_problem(prob)
    Ud = to_dev(U)
    s.step(Ud, s.max_dt(Ud, 0.5), 2)
    dt = 0.8 * s.max_dt(Ud, 0.5)
    lam = to_dev(np.random.default_rng(4).standard_normal(U.shape))
    l_ref, p_ref = s.step_vjp(Ud, dt, lam)
    G = _group(B, prob, world, ov)
    L, p = G.step_vjp(G.scatter(Ud), dt, G.scatter(lam))
    out = G.gather(L)
    assert float((out - l_ref).abs().max()) <= 1e-12 * float(l_ref.abs().max())
    nz = p_ref.abs() > 0
    assert bool(nz[0]) and torch.equal(nz, p.abs() > 0)
    assert float((p - p_ref).abs().max()) <= 1e-12 * float(p_ref.abs().max())


def test_slab_overlap_too_shallow_for_the_body(env):
    torch, B = env
    prob, _ = _cylinder()
    with pytest.raises(B.JsError) as e:
        B.Solver.slab(prob, 15, 15, 3)  # the cylinder (rows 13..31) crosses rows 15 and 30
    assert e.value.code == B.JS_ERR_IB
    sl = B.Solver.slab(prob, 15, 15, 14)
    assert sl.window == (1, 43, 14, 15)


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob, U = _cylinder()
        plan = parallel.SlabPlan(prob.ny, world, 14)
        G = parallel.SlabGroup.build(prob, plan, [rank], parallel.DistTransport())
        X = G.scatter(to_dev(U))
        dts = []
        for _ in range(4):
            dt = G.max_dt(X, 0.5)
            dts.append(dt)
            G.step(X, dt, 1)
        lam = to_dev(np.random.default_rng(4).standard_normal(U.shape))
        L, p = G.step_vjp(X, 0.8 * dts[-1], G.scatter(lam))
        q.put((rank, to_host(G.gather(X)), dts, to_host(G.gather(L)), to_host(p)))
    finally:
        dist.destroy_process_group()


def test_two_processes_gloo_exchange_equal_whole_grid(env):
    torch, B = env
    import torch.multiprocessing as mp
    world = 2
    port = 29700 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    prob, U = _cylinder()
    s = B.Solver.from_problem(prob)
    Ud = to_dev(U)
    dts = []
    for _ in range(4):
        dts.append(s.max_dt(Ud, 0.5))
        s.step(Ud, dts[-1], 1)
    lam = to_dev(np.random.default_rng(4).standard_normal(U.shape))
    l_ref, p_ref = s.step_vjp(Ud, 0.8 * dts[-1], lam)
    plan = parallel.SlabPlan(prob.ny, world, 14)
    out, lo = np.zeros(U.shape), np.zeros(U.shape)
    for rank, x, d, l, p in res:
        assert d == dts
        rows = slice(plan.row0[rank], plan.row0[rank] + plan.nrows[rank])
        out[:, rows] = x[:, rows]
        lo[:, rows] = l[:, rows]
        pr = to_host(p_ref)
        assert np.abs(p - pr).max() <= 1e-12 * np.abs(pr).max()
    assert np.array_equal(out, to_host(Ud))
    lr = to_host(l_ref)
    assert np.abs(lo - lr).max() <= 1e-12 * np.abs(lr).max()


def test_full_size_cylinder_in_four_slabs(env):
    """The 2048 x 1024 viscous shock-cylinder configuration (inflow, outflow, reflective walls, the
    immersed cylinder centred on the middle slab boundary) in 4 slabs of 256 rows: 10 steps equal
    to the whole grid bit for bit, and one reverse step equal to js_step_vjp to 1e-12."""
    torch, B = env
    prob = W.shock_cylinder()
    s = B.Solver.from_problem(prob)
    Ud = s.prim_to_cons(torch.tensor(prob.W0, device="cuda"))
    G = _group(B, prob, 4, 14)
    X = G.scatter(Ud)
    for _ in range(10):
        dt = s.max_dt(Ud, 0.5)
        assert G.max_dt(X, 0.5) == dt
        s.step(Ud, dt, 1)
        G.step(X, dt, 1)
    assert torch.equal(G.gather(X), Ud)
    lam = torch.randn_like(Ud)
    dt = 0.8 * s.max_dt(Ud, 0.5)
    l_ref, p_ref = s.step_vjp(Ud, dt, lam)
    L, p = G.step_vjp(G.scatter(Ud), dt, G.scatter(lam))
    assert float((G.gather(L) - l_ref).abs().max()) <= 1e-12 * float(l_ref.abs().max())
    assert float((p - p_ref).abs().max()) <= 1e-12 * float(p_ref.abs().max())
    assert s.status() == 0 and all(sl.status() == 0 for sl in G.slabs.values())
