"""The CFL step of js_max_dt against the oracle's, bit for bit, on states built to stress the
two-pass reduction (the fast pass-1 rate and its IEEE pass-2 candidates): a near-vacuum,
hypersonic cell (E/p up to 1e12, where the fast rate's error bound fails and pass 1 must take
the IEEE rate itself) holding the maximum at a row start, a warp boundary and a block boundary;
uniform runs of the maximum-rate state crossing warp, block and row boundaries; and
non-physical cells (negative density or pressure, NaN), which must be reported as
JS_ERR_NONPHYSICAL (the oracle's step rejects such states)."""
import numpy as np
import pytest

import oracle as O
from paper_2601_04400_gb300 import workloads as W
from jsutil import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04400_gb300 import binding
    binding.lib()
    return binding


def _base(nx, ny, mu=0.0):
    p = W.riemann2d(nx, ny=ny).with_(mu=mu)
    Wp = W.random_state(p.with_(W0=np.stack([np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)),
                                             np.ones((ny, nx))])), seed=5, amp=0.1)
    return p, Wp


def _cons(p, Wp):
    return O.prim_to_cons(p, Wp)


@pytest.mark.parametrize("mu", [0.0, 2e-3])
@pytest.mark.parametrize("cell", [(3, 0), (0, 31), (0, 32), (2, 55), (2, 56), (7, 99)])
@pytest.mark.parametrize("e_over_p", [1e6, 1e9, 1e12])
def test_hypersonic_near_vacuum_cell_holds_the_maximum(B, mu, cell, e_over_p):
    """One cell with E/p = e_over_p and the largest rate; grid 100 x 40 (rows do not align with
    warps or blocks).  Cells (j, i) are chosen at a row start, around lanes 31/32 of a warp and
    across the 256-cell block boundary (flat index 255/256)."""
    nx, ny = 100, 40
    p, Wp = _base(nx, ny, mu)
    j, i = cell
    u = 20.0
    Wp[:, j, i] = (1.0, u, 0.3, 0.5 * u * u * 0.4 / e_over_p)
    U = _cons(p, Wp)
    s = B.Solver.from_problem(p)
    assert s.max_dt(to_dev(U), 0.5) == O.max_dt(p, U, 0.5)
    s.close()


@pytest.mark.parametrize("start,length", [(250, 40), (95, 300), (31, 2), (600, 1000), (0, 4000)])
def test_uniform_run_of_the_maximum_crosses_warps_blocks_and_rows(B, start, length):
    """The maximum-rate state fills cells start .. start+length-1 (flat index, row-major, 100
    cells per row): pass 2 takes its IEEE rate once per run along a row; the result must still
    be the one-pass maximum.  A second, slightly slower run elsewhere competes."""
    nx, ny = 100, 48
    p, Wp = _base(nx, ny)
    flat = Wp.reshape(4, -1)
    flat[:, start:start + length] = np.array([0.7, 3.0, -1.5, 2.0])[:, None]
    flat[:, 4500:4530] = np.array([0.7, 2.9999999999, -1.5, 2.0])[:, None]
    U = _cons(p, Wp)
    s = B.Solver.from_problem(p)
    assert s.max_dt(to_dev(U), 0.5) == O.max_dt(p, U, 0.5)
    s.close()


def test_near_ties_are_resolved_like_the_oracle(B):
    """Many cells whose rates agree to within a few ulp: the IEEE maximum decides."""
    nx, ny = 300, 300
    p, Wp = _base(nx, ny)
    rng = np.random.default_rng(3)
    Wp[1] = 2.0 * (1.0 + rng.integers(-4, 5, (ny, nx)) * 2.0 ** -52)
    Wp[2] = 0.0
    Wp[0] = 1.0
    Wp[3] = 1.0
    U = _cons(p, Wp)
    s = B.Solver.from_problem(p)
    assert s.max_dt(to_dev(U), 0.5) == O.max_dt(p, U, 0.5)
    s.close()


@pytest.mark.parametrize("mu", [0.0, 2e-3])
@pytest.mark.parametrize("bad", ["negative_density", "negative_pressure", "nan_momentum", "zero_density"])
def test_non_physical_cell_is_reported(B, mu, bad):
    nx, ny = 100, 40
    p, Wp = _base(nx, ny, mu)
    U = _cons(p, Wp)
    j, i = 17, 63
    if bad == "negative_density":
        U[0, j, i] = -0.5
    elif bad == "negative_pressure":
        U[3, j, i] = 0.0
        U[1, j, i] = 1.0
    elif bad == "nan_momentum":
        U[2, j, i] = np.nan
    else:
        U[0, j, i] = 0.0
    s = B.Solver.from_problem(p)
    with pytest.raises(B.JsError) as e:
        s.max_dt(to_dev(U), 0.5)
    assert e.value.code == B.JS_ERR_NONPHYSICAL
    s.close()


# ---------------------------------------------------------------------------------------
# js_step_cfl: the CFL step size computed on the device, no host synchronisation
# ---------------------------------------------------------------------------------------
def _host_loop(s, U, cfl, n, t_end=None):
    dts, t = [], 0.0
    for _ in range(n):
        if t_end is not None and not t < t_end:
            break
        dt = s.max_dt(U, cfl)
        if t_end is not None and t + dt > t_end:
            dt = t_end - t
        s.step(U, dt, 1)
        t = t + dt
        dts.append(dt)
    return np.array(dts), t


@pytest.mark.parametrize("prob", [W.riemann2d(96, ny=70), W.shock_cylinder(nx=128, ny=64), W.sod(200)],
                         ids=["four_quadrant_96x70", "viscous_cylinder_128x64", "sod200"])
def test_device_cfl_steps_equal_host_cfl_steps(B, prob):
    import torch
    U0 = O.prim_to_cons(prob, prob.W0)
    s = B.Solver.from_problem(prob)
    Ua, Ub = to_dev(U0), to_dev(U0)
    dts_h, _ = _host_loop(s, Ua, prob.cfl, 25)
    log = torch.zeros(25, dtype=torch.float64, device="cuda")
    t = torch.zeros((), dtype=torch.float64, device="cuda")
    s.step_cfl(Ub, prob.cfl, 25, t=t, dt_log=log)
    assert s.status() == 0
    assert log.cpu().numpy().tobytes() == dts_h.tobytes()
    assert Ua.cpu().numpy().tobytes() == Ub.cpu().numpy().tobytes()
    t_h = 0.0
    for dt in dts_h.tolist():
        t_h = t_h + dt  # the device accumulates t = t + dt in step order
    assert float(t) == t_h
    s.close()


def test_device_cfl_steps_stop_at_the_end_time(B):
    """Four-quadrant 96^2 to t = 0.05 in one call with more steps than needed: the last step is
    clipped, the rest do nothing.  The step sizes equal those of the host loop (js_max_dt, the
    same clipping) bit for bit, the state equals that loop's, and the oracle's run to the same
    time agrees within the parity bar."""
    import torch
    p = W.riemann2d(96)
    U0 = O.prim_to_cons(p, p.W0)
    t_end = 0.05
    Uo, dts_o = O.run_to(p, U0, p.cfl, t_end)
    s = B.Solver.from_problem(p)
    Uh = to_dev(U0)
    dts_h, t_h = _host_loop(s, Uh, p.cfl, 10 ** 6, t_end=t_end)
    assert len(dts_h) == len(dts_o) and t_h == t_end
    U = to_dev(U0)
    n = len(dts_h) + 7
    log = torch.zeros(n, dtype=torch.float64, device="cuda")
    t = torch.zeros((), dtype=torch.float64, device="cuda")
    s.step_cfl(U, p.cfl, n, t=t, t_end=t_end, dt_log=log)
    assert s.status() == 0
    lg = log.cpu().numpy()
    assert lg[:len(dts_h)].tobytes() == dts_h.tobytes() and (lg[len(dts_h):] == 0).all()
    assert float(t) == t_end
    assert U.cpu().numpy().tobytes() == Uh.cpu().numpy().tobytes()
    from jsutil import TOL, normwise_err
    assert normwise_err(U.cpu().numpy(), Uo) < TOL
    s.close()


def test_device_cfl_steps_in_ieee_mode_are_the_oracle_run_bit_for_bit(B):
    import torch
    p = W.shock_cylinder(nx=128, ny=64)
    U0 = O.prim_to_cons(p, p.W0)
    Uo, dts_o = O.run_to(p, U0, p.cfl, 1e9, max_steps=60)
    s = B.Solver.from_problem(p)
    s.set_arith("ieee")
    U = to_dev(U0)
    log = torch.zeros(60, dtype=torch.float64, device="cuda")
    s.step_cfl(U, p.cfl, 60, dt_log=log)
    assert s.status() == 0
    assert log.cpu().numpy().tobytes() == dts_o.tobytes()
    assert U.cpu().numpy().tobytes() == Uo.tobytes()
    s.close()


def test_device_cfl_steps_capture_into_a_cuda_graph(B):
    import torch
    p = W.shock_cylinder(nx=160, ny=96)
    U0 = O.prim_to_cons(p, p.W0)
    stream = torch.cuda.Stream()
    s = B.Solver.from_problem(p, stream=stream)
    ref = to_dev(U0)
    with torch.cuda.stream(stream):
        s.step_cfl(ref, p.cfl, 12)
    stream.synchronize()
    U = to_dev(U0)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        s.step_cfl(U, p.cfl, 4)
    U.copy_(to_dev(U0))
    torch.cuda.synchronize()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert s.status() == 0
    assert U.cpu().numpy().tobytes() == ref.cpu().numpy().tobytes()
    s.close()


def test_device_cfl_step_of_a_non_physical_state_does_nothing(B):
    p = W.riemann2d(64)
    U0 = O.prim_to_cons(p, p.W0)
    U0[0, 20, 30] = -1.0
    s = B.Solver.from_problem(p)
    U = to_dev(U0)
    s.step_cfl(U, p.cfl, 3)
    assert s.status() == B.JS_ERR_NONPHYSICAL
    assert U.cpu().numpy().tobytes() == U0.tobytes()
    s.close()
