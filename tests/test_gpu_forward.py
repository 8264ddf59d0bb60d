"""Parity of the CUDA forward path (js_rhs, js_step, js_max_dt, js_prim_to_cons) with the
FP64 oracle, element by element, on seeded inputs shaped like the paper's cases: tiny and
ragged grids that span several tiles, every boundary kind, the immersed cylinder, and the
full-size four-quadrant and shock-cylinder grids."""
import numpy as np
import pytest

import oracle as O
from paper_2601_04400_gb300 import workloads as W
from jsutil import TOL, normwise_err, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04400_gb300 import binding
    binding.lib()
    return binding


def _cases():
    """(name, problem, primitive state) covering 1D/2D, ragged sizes, boundaries, NS, IB."""
    out = []
    p = W.sod(200)
    out.append(("sod200", p, p.W0))
    p = W.riemann2d(70, ny=45)
    out.append(("riemann_ragged_70x45", p, p.W0))
    p = W.random_periodic(96, 40, seed=3, mu=3e-3, nu=2e-4)
    out.append(("periodic_ns_av_96x40", p, p.W0))
    p = W.shock_cylinder(nx=100, ny=52, mach=2.0, Re=500.0)
    out.append(("cylinder_ns_100x52", p, W.random_state(p, seed=2, amp=0.02)))
    p = W.shock_cylinder(nx=64, ny=40, mach=2.5, viscous=False)
    out.append(("cylinder_euler_64x40", p, W.random_state(p, seed=5, amp=0.05)))
    # the unperturbed initial condition: the quiescent gas ahead of the shock gives contact
    # speed s* = 0 exactly at most faces (the two-branch average of the HLLC flux)
    p = W.shock_cylinder(nx=100, ny=52, mach=2.0, Re=500.0)
    out.append(("cylinder_ns_initial_100x52", p, p.W0))
    p = W.random_periodic(33, 38, seed=9).with_(bc=(1, 3, 3, 1), inflow=np.array(
        [[1.1, 0.2, 0.1, 0.9], [0.9, -0.1, 0.0, 1.1], [1.0, 0.05, 0.3, 1.0], [1.2, 0.0, -0.2, 0.8]]))
    out.append(("mixed_bc_33x38", p, p.W0))
    p = W.random_periodic(40, 24, seed=4).with_(bc=(0, 0, 1, 1), wall=1, mu=1e-3)
    out.append(("refl_noslipflag_40x24", p, p.W0))
    return out


CASES = _cases()


@pytest.mark.parametrize("name,prob,Wp", CASES, ids=[c[0] for c in CASES])
def test_prim_to_cons_matches_oracle(B, name, prob, Wp):
    s = B.Solver.from_problem(prob)
    U = to_host(s.prim_to_cons(to_dev(Wp)))
    assert normwise_err(U, O.prim_to_cons(prob, Wp)) < 1e-15


@pytest.mark.parametrize("name,prob,Wp", CASES, ids=[c[0] for c in CASES])
def test_max_dt_is_bit_exact(B, name, prob, Wp):
    U = O.prim_to_cons(prob, Wp)
    s = B.Solver.from_problem(prob)
    assert s.max_dt(to_dev(U), 0.5) == O.max_dt(prob, U, 0.5)


@pytest.mark.parametrize("name,prob,Wp", CASES, ids=[c[0] for c in CASES])
def test_rhs_matches_oracle(B, name, prob, Wp):
    U = O.prim_to_cons(prob, Wp)
    s = B.Solver.from_problem(prob)
    L = to_host(s.rhs(to_dev(U)))
    assert s.status() == 0
    ref = O.rhs(prob, U)
    assert normwise_err(L, ref) < TOL


@pytest.mark.parametrize("name,prob,Wp", CASES, ids=[c[0] for c in CASES])
def test_steps_match_oracle(B, name, prob, Wp):
    U0 = O.prim_to_cons(prob, Wp)
    s = B.Solver.from_problem(prob)
    dt = 0.8 * O.max_dt(prob, U0, 0.5)
    Ud = to_dev(U0)
    Uo = U0
    for n in (1, 9, 20):  # cumulative 1, 10, 30 steps
        s.step(Ud, dt, n)
        Uo = O.step(prob, Uo, [dt] * n)
        assert normwise_err(to_host(Ud), Uo) < TOL, n
    assert s.status() == 0


def test_sod_full_run_matches_oracle_and_exact(B):
    p = W.sod(200)
    U0 = O.prim_to_cons(p, p.W0)
    Uo, dts = O.run_to(p, U0, p.cfl, p.t_end)
    s = B.Solver.from_problem(p)
    Ud = to_dev(U0)
    for dt in dts:
        # the GPU's own CFL step on its own state agrees with the oracle's sequence
        s.step(Ud, dt, 1)
    Ug = to_host(Ud)
    assert normwise_err(Ug, Uo) < TOL
    x = (np.arange(200) + 0.5) / 200
    r, _, _, _ = O.exact_riemann((1, 0, 1), (0.125, 0, 0.1), 1.4, x, 0.5, 0.2)
    assert np.mean(np.abs(Ug[0, 0] - r)) < 3e-3


def test_gpu_cfl_sequence_matches_oracle_on_sod(B):
    p = W.sod(200)
    U0 = O.prim_to_cons(p, p.W0)
    _, dts = O.run_to(p, U0, p.cfl, p.t_end)
    s = B.Solver.from_problem(p)
    Ud = to_dev(U0)
    t, k = 0.0, 0
    while t < p.t_end:
        dt = s.max_dt(Ud, p.cfl)
        if t + dt > p.t_end:
            dt = p.t_end - t
        assert abs(dt - dts[k]) <= 1e-12 * dts[k]
        s.step(Ud, dt, 1)
        t += dt
        k += 1
    assert k == len(dts)


def test_ib_tables_match_oracle(B):
    for prob in (W.shock_cylinder(nx=256, ny=128), W.adjoint_case(128), W.batched_cases(3, seed=1)[2]):
        s = B.Solver.from_problem(prob)
        n, tag = s.ib_info()
        t = O.ib_tables(prob)
        assert n == len(t["gcell"])
        assert np.array_equal(tag, t["tag"])


def test_nonphysical_state_sets_the_error_flag(B):
    p = W.riemann2d(64)
    Wp = np.array(p.W0)
    Wp[3, 10, 20] = -0.5  # negative pressure in one fluid cell
    s = B.Solver.from_problem(p)
    Ud = s.prim_to_cons(to_dev(Wp))
    s.step(Ud, 1e-5, 1)
    assert s.status() == B.JS_ERR_NONPHYSICAL
    assert s.status() == 0  # the flag is cleared by reading it


def test_step_is_graph_capturable(B):
    import torch
    p = W.riemann2d(80, ny=72)
    Wp = W.random_state(p, seed=1)
    U0 = O.prim_to_cons(p, Wp)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        s = B.Solver.from_problem(p, stream=side)
        Ug = to_dev(U0)
        s.step(Ug.clone(), 1e-4, 1)  # warm-up outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            s.step(Ug, 1e-4, 2)
    torch.cuda.synchronize()
    Ug.copy_(to_dev(U0))
    torch.cuda.synchronize()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    ref = O.step(p, U0, [1e-4] * 4)
    assert normwise_err(to_host(Ug), ref) < TOL


@pytest.mark.parametrize("which", ["riemann2d_1024", "shock_cylinder_2048x1024", "mach5_cylinder_4347x1932"])
def test_full_size_matches_oracle(B, which):
    """Full-size grids: 3 steps from the initial state, then one step from a GPU state
    evolved further, compared with the oracle on every cell.  The paper's Mach-5 cylinder
    grid (8.4e6 cells) is ragged in both directions."""
    p = {"riemann2d_1024": lambda: W.riemann2d(1024), "shock_cylinder_2048x1024": W.shock_cylinder,
         "mach5_cylinder_4347x1932": W.mach5_cylinder}[which]()
    U0 = O.prim_to_cons(p, p.W0)
    dt = O.max_dt(p, U0, p.cfl)
    s = B.Solver.from_problem(p)
    Ud = to_dev(U0)
    s.step(Ud, dt, 3)
    assert normwise_err(to_host(Ud), O.step(p, U0, [dt] * 3)) < TOL
    s.step(Ud, dt, 40)
    Ug = to_host(Ud)
    dt2 = s.max_dt(Ud, p.cfl)
    assert dt2 == O.max_dt(p, Ug, p.cfl)
    s.step(Ud, dt2, 1)
    assert normwise_err(to_host(Ud), O.step(p, Ug, [dt2])) < TOL
    assert s.status() == 0


def test_every_tile_variant_gives_identical_results(B):
    for prob in (W.riemann2d(100, ny=70), W.shock_cylinder(nx=130, ny=66)):
        U0 = O.prim_to_cons(prob, W.random_state(prob, seed=8, amp=0.02))
        s = B.Solver.from_problem(prob)
        dt = 0.5 * s.max_dt(to_dev(U0), 0.5)
        _, n = s.tuning()
        assert n >= 2
        res = []
        for v in range(n):
            s.set_tuning(v)
            Ud = to_dev(U0)
            s.step(Ud, dt, 3)
            res.append(to_host(Ud))
            Lr = to_host(s.rhs(to_dev(U0)))
            res.append(Lr)
        for v in range(1, n):
            assert np.array_equal(res[2 * v], res[0]), v
            assert np.array_equal(res[2 * v + 1], res[1]), v
        assert s.status() == 0
