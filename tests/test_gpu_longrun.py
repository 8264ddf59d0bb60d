"""Parity over the benchmark configurations' full step counts, on reduced grids the oracle
finishes in seconds: the four-quadrant Riemann problem to t = 0.8 with the CFL rule, and the
viscous shock-cylinder case over 2000 steps.  The GPU computes its own CFL steps; they must
equal the oracle's sequence, and the final states must agree to the parity bar."""
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


def _gpu_run_to(B, prob, U0, cfl, t_end, max_steps):
    s = B.Solver.from_problem(prob)
    Ud = to_dev(U0)
    t, dts = 0.0, []
    while t < t_end and len(dts) < max_steps:
        dt = s.max_dt(Ud, cfl)
        if t + dt > t_end:
            dt = t_end - t
        s.step(Ud, dt, 1)
        t += dt
        dts.append(dt)
    assert s.status() == 0
    return to_host(Ud), np.array(dts)


def test_four_quadrant_to_t08_matches_oracle(B):
    p = W.riemann2d(96)
    U0 = O.prim_to_cons(p, p.W0)
    Uo, dts_o = O.run_to(p, U0, p.cfl, p.t_end)
    Ug, dts_g = _gpu_run_to(B, p, U0, p.cfl, p.t_end, 100000)
    assert len(dts_g) == len(dts_o) and len(dts_o) > 500
    assert np.abs(dts_g - dts_o).max() <= 1e-11 * dts_o.max()
    assert normwise_err(Ug, Uo) < TOL


def test_viscous_cylinder_2000_steps_matches_oracle(B):
    p = W.shock_cylinder(nx=128, ny=64)
    U0 = O.prim_to_cons(p, p.W0)
    n = p.n_steps
    Uo, dts_o = O.run_to(p, U0, p.cfl, 1e9, max_steps=n)
    Ug, dts_g = _gpu_run_to(B, p, U0, p.cfl, 1e9, n)
    assert len(dts_o) == len(dts_g) == n
    assert np.abs(dts_g - dts_o).max() <= 1e-11 * dts_o.max()
    assert normwise_err(Ug, Uo) < TOL
