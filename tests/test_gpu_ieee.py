"""The IEEE-order arithmetic mode (js_set_arith(ctx, JS_ARITH_IEEE)) equals the oracle BIT FOR
BIT: both evaluate every formula of the right-hand side, the immersed-boundary fill and the
Runge-Kutta stage as single IEEE-rounded double operations in the same canonical order (the
oracle is plain C++ compiled without contraction), so no rounding difference can arise and
chaotic flows stay identical over any number of steps.  Cases: every forward-parity problem
(1D, ragged 2D, periodic NS with artificial viscosity, NS and Euler cylinders, mixed and
reflective boundaries, the no-slip flag), the oblique wall, states where the positivity fallback
acts, and CFL-driven runs."""
import numpy as np
import pytest

import oracle as O
from paper_2601_04400_gb300 import workloads as W
from jsutil import to_dev, to_host
from test_gpu_forward import CASES
from test_gpu_pins import _oblique_wall, _rough

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04400_gb300 import binding
    binding.lib()
    return binding


def _solver(B, prob):
    s = B.Solver.from_problem(prob)
    s.set_arith("ieee")
    assert s.arith() == "ieee"
    return s


def _same(a, b):
    """Bitwise equality (NaN-free arrays; -0.0 and 0.0 are told apart)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return a.shape == b.shape and a.tobytes() == b.tobytes()


def _ndiff(a, b):
    return int((np.ascontiguousarray(a).view(np.int64) != np.ascontiguousarray(b).view(np.int64)).sum())


EXTRA = []
for _n, _mu, _wall in ((64, 0.0, 0), (70, 2e-3, 1)):
    _p, _Wp = _oblique_wall(_n, _mu)
    EXTRA.append(("oblique_wall_%d_mu%g_wall%d" % (_n, _mu, _wall), _p.with_(wall=_wall), _Wp))
_p = W.mach5_cylinder(nx=218, ny=97)
EXTRA.append(("mach5_218x97", _p, _p.W0))
ALL = CASES + EXTRA


@pytest.mark.parametrize("name,prob,Wp", ALL, ids=[c[0] for c in ALL])
def test_rhs_is_bitwise_the_oracle(B, name, prob, Wp):
    U = O.prim_to_cons(prob, Wp)
    s = _solver(B, prob)
    L = to_host(s.rhs(to_dev(U)))
    assert s.status() == 0
    ref = O.rhs(prob, U)
    assert _same(L, ref), "%d of %d values differ" % (_ndiff(L, ref), L.size)
    s.close()


@pytest.mark.parametrize("name,prob,Wp", ALL, ids=[c[0] for c in ALL])
def test_steps_are_bitwise_the_oracle(B, name, prob, Wp):
    U0 = O.prim_to_cons(prob, Wp)
    s = _solver(B, prob)
    dt = 0.8 * O.max_dt(prob, U0, 0.5)
    Ud = to_dev(U0)
    Uo = U0
    for n in (1, 9, 20):  # cumulative 1, 10, 30 steps
        s.step(Ud, dt, n)
        Uo = O.step(prob, Uo, [dt] * n)
        got = to_host(Ud)
        assert _same(got, Uo), "after %d more steps: %d values differ" % (n, _ndiff(got, Uo))
    assert s.status() == 0
    s.close()


@pytest.mark.parametrize("nx,ny", [(200, 1), (64, 48), (37, 70)])
def test_rhs_with_fallback_faces_is_bitwise_the_oracle(B, nx, ny):
    p, Wp = _rough(nx, ny, 7)
    U = O.prim_to_cons(p, Wp)
    s = _solver(B, p)
    got = to_host(s.rhs(to_dev(U)))
    ref = O.rhs(p, U)
    assert _same(got, ref), "%d values differ" % _ndiff(got, ref)
    s.close()


def _cfl_run_both(B, p, U0, t_end, max_steps):
    """The GPU's own CFL steps (js_max_dt, last one clipped as the oracle clips it) in IEEE
    mode, and the oracle's run_to."""
    Uo, dts_o = O.run_to(p, U0, p.cfl, t_end, max_steps=max_steps)
    s = _solver(B, p)
    Ud = to_dev(U0)
    t, dts = 0.0, []
    while t < t_end and len(dts) < max_steps:
        dt = s.max_dt(Ud, p.cfl)
        if t + dt > t_end:
            dt = t_end - t
        s.step(Ud, dt, 1)
        t = t + dt
        dts.append(dt)
    assert s.status() == 0
    got = to_host(Ud)
    s.close()
    return got, Uo, np.array(dts), dts_o


def test_sod_to_t02_is_bitwise_the_oracle(B):
    p = W.sod(200)
    got, ref, dts, dts_o = _cfl_run_both(B, p, O.prim_to_cons(p, p.W0), p.t_end, 10 ** 6)
    assert _same(dts, dts_o) and _same(got, ref)


def test_four_quadrant_96_to_t08_is_bitwise_the_oracle(B):
    p = W.riemann2d(96)
    got, ref, dts, dts_o = _cfl_run_both(B, p, O.prim_to_cons(p, p.W0), p.t_end, 10 ** 6)
    assert len(dts) > 500
    assert _same(dts, dts_o) and _same(got, ref), _ndiff(got, ref)


def test_viscous_cylinder_128x64_2000_steps_is_bitwise_the_oracle(B):
    p = W.shock_cylinder(nx=128, ny=64)
    got, ref, dts, dts_o = _cfl_run_both(B, p, O.prim_to_cons(p, p.W0), 1e9, p.n_steps)
    assert len(dts) == p.n_steps
    assert _same(dts, dts_o) and _same(got, ref), _ndiff(got, ref)


def test_mode_switch_and_neural_flux_are_exclusive(B):
    import torch
    p = W.riemann2d(48)
    s = B.Solver.from_problem(p)
    U = to_dev(O.prim_to_cons(p, p.W0))
    fast = to_host(s.rhs(U))
    s.set_arith("ieee")
    ieee = to_host(s.rhs(U))
    s.set_arith("fast")
    assert _same(to_host(s.rhs(U)), fast)
    assert np.abs(ieee - fast).max() <= 1e-12 * np.abs(fast).max()
    from paper_2601_04400_gb300 import neural as NN
    w = NN.init_weights(0)
    s.set_neural(w, NN.frame_norm(U, scale=0.1))
    s.set_arith("ieee")
    with pytest.raises(B.JsError) as e:
        s.rhs(U)
    assert e.value.code == B.JS_ERR_ARG
    s.set_neural(None)
    torch.cuda.synchronize()
    s.close()
