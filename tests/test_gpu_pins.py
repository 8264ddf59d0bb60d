"""GPU parity on the cases whose oracle behaviour the CPU pins fix independently
(tests/test_oracle_pins.py): the immersed boundary on an oblique (30 degree) slip wall, and the
positivity fallback of the face states (first-order cell states where a WENO5-reconstructed
density or pressure is not positive).  The GPU must take the fallback at the same faces: its
RHS and steps equal the oracle's within the parity bar on states where the oracle counts
fallback faces."""
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


def _oblique_wall(n, mu=0.0, seed=0):
    th = np.pi / 6
    t = np.array([np.cos(th), np.sin(th)])
    nrm = np.array([-np.sin(th), np.cos(th)])
    X, Y = W.cell_centres(n, n, 0.0, 0.0, 1.0 / n, 1.0 / n)
    sdf = (X - 0.3) * nrm[0] + Y * nrm[1]
    p = W.riemann2d(n).with_(sdf=sdf, mu=mu)
    Wp = np.zeros((4, n, n))
    Wp[0], Wp[1], Wp[2], Wp[3] = 1.3, 0.7 * t[0] + 0.2 * X, 0.7 * t[1] - 0.1 * Y, 0.9 + 0.1 * X
    Wp = W.random_state(p.with_(W0=Wp), seed=seed, amp=0.03)
    solid = sdf < 0
    for c, v in enumerate((5.0, -3.0, 2.0, 7.0)):
        Wp[c][solid] = v
    return p, Wp


@pytest.mark.parametrize("n,mu,wall", [(64, 0.0, 0), (96, 2e-3, 0), (70, 2e-3, 1)])
def test_oblique_wall_matches_oracle(B, n, mu, wall):
    p, Wp = _oblique_wall(n, mu)
    p = p.with_(wall=wall)
    U0 = O.prim_to_cons(p, Wp)
    s = B.Solver.from_problem(p)
    assert normwise_err(to_host(s.rhs(to_dev(U0))), O.rhs(p, U0)) < TOL
    dt = O.max_dt(p, U0, 0.5)
    Ud = to_dev(U0)
    s.step(Ud, dt, 10)
    assert s.status() == 0
    assert normwise_err(to_host(Ud), O.step(p, U0, [dt] * 10)) < TOL
    s.close()


def _rough(nx, ny, seed):
    rng = np.random.default_rng(seed)
    p = (W.riemann2d(nx, ny=ny) if ny > 1 else W.sod(nx)).with_(name="rough")
    Wp = np.zeros((4, ny, nx))
    Wp[0] = 10 ** rng.uniform(-2, 1, (ny, nx))
    Wp[1] = rng.uniform(-1, 1, (ny, nx))
    if ny > 1:
        Wp[2] = rng.uniform(-0.5, 0.5, (ny, nx))
    Wp[3] = 10 ** rng.uniform(-4, 2, (ny, nx))
    return p, Wp


@pytest.mark.parametrize("nx,ny", [(200, 1), (64, 48), (37, 70)])
def test_rhs_with_many_fallback_faces_matches_oracle(B, nx, ny):
    """Rough states (density over 3, pressure over 6 decades): a third of the faces take the
    fallback.  The RHS is compared where it is finite on both sides (every cell here)."""
    p, Wp = _rough(nx, ny, 7)
    U = O.prim_to_cons(p, Wp)
    O.fallback_faces()
    ref = O.rhs(p, U)
    assert O.fallback_faces() > (nx * ny) // 10
    s = B.Solver.from_problem(p)
    got = to_host(s.rhs(to_dev(U)))
    assert s.status() == 0
    assert normwise_err(got, ref) < TOL
    s.close()


def _run_both(B, p, U0, n_steps):
    Uo, dts = O.run_to(p, U0, p.cfl, 1e9, max_steps=n_steps)
    s = B.Solver.from_problem(p)
    Ud = to_dev(U0)
    for dt in dts:
        s.step(Ud, dt, 1)
    assert s.status() == 0
    got = to_host(Ud)
    s.close()
    return got, Uo


def test_mach5_cylinder_first_steps_with_fallback_match_oracle(B):
    """The paper's Mach-5 shock-cylinder case (Euler, immersed cylinder) at 218 x 97: the
    oracle already takes the fallback at three faces in the first step."""
    p = W.mach5_cylinder(nx=218, ny=97)
    U0 = O.prim_to_cons(p, p.W0)
    O.fallback_faces()
    got, ref = _run_both(B, p, U0, 20)
    assert O.fallback_faces() > 0
    assert normwise_err(got, ref) < TOL


def test_blast_wave_2d_through_the_fallback_matches_oracle(B):
    """A circular blast (p = 1000 inside radius 0.1, 0.01 outside) in a reflective box, 96^2:
    the oracle's first fallback faces appear at step 131; 140 CFL steps compared."""
    n = 96
    p = W.riemann2d(n).with_(bc=(1, 1, 1, 1), name="blast2d")
    X, Y = W.cell_centres(n, n, 0.0, 0.0, 1.0 / n, 1.0 / n)
    Wp = np.zeros((4, n, n))
    Wp[0] = 1.0
    Wp[3] = np.where((X - 0.3) ** 2 + (Y - 0.4) ** 2 < 0.01, 1000.0, 0.01)
    U0 = O.prim_to_cons(p, Wp)
    O.fallback_faces()
    got, ref = _run_both(B, p, U0, 140)
    assert O.fallback_faces() > 0
    assert normwise_err(got, ref) < TOL


def test_blast_wave_1d_through_the_fallback_matches_oracle(B):
    """Two interacting blast waves (1000 | 0.01 | 100, reflective ends), 400 cells, 960 CFL
    steps (the oracle's first fallback faces are at step 942)."""
    n = 400
    p = W.sod(n).with_(name="blast", bc=(1, 1, 0, 0))
    x = (np.arange(n) + 0.5) / n
    Wp = np.zeros((4, 1, n))
    Wp[0] = 1.0
    Wp[3, 0] = np.where(x < 0.1, 1000.0, np.where(x < 0.9, 0.01, 100.0))
    U0 = O.prim_to_cons(p, Wp)
    O.fallback_faces()
    got, ref = _run_both(B, p, U0, 960)
    assert O.fallback_faces() > 0
    assert normwise_err(got, ref) < TOL
