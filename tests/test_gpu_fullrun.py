"""Parity at the benchmark configurations' full sizes AND full step counts: the 1024x1024
four-quadrant Riemann problem to t = 0.8 with the CFL rule (about 7,100 steps) and the
2048x1024 viscous Mach-2 shock-cylinder case over 2000 steps.  The GPU takes its own CFL
steps (js_max_dt + js_step); the oracle advances the same grid with its own.  States are
compared at checkpoints; the step sizes and the final states must agree to the parity bar.

The oracle needs tens of CPU minutes for these, so they run only with JS_FULLRUN=1 (and
carry no `gpu` marker: the routine GPU suite leaves them out)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2601_04400_gb300 import workloads as W
from jsutil import TOL, normwise_err, to_dev, to_host

pytestmark = [pytest.mark.fullrun,
              pytest.mark.skipif(os.environ.get("JS_FULLRUN") != "1", reason="set JS_FULLRUN=1 to run")]

CHUNK = 500


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04400_gb300 import binding
    binding.lib()
    return binding


def _run_both(B, prob, t_end, max_steps):
    """Advance GPU and oracle side by side in chunks; returns per-checkpoint errors."""
    U0 = O.prim_to_cons(prob, prob.W0)
    s = B.Solver.from_problem(prob)
    Ud = to_dev(U0)
    Uo = U0
    t, n, hist, max_ddt = 0.0, 0, [], 0.0
    while t < t_end and n < max_steps:
        k = min(CHUNK, max_steps - n)
        # oracle: k CFL steps (the last one clipped to t_end)
        Uo, dts_o = O.run_to(prob, Uo, prob.cfl, t_end - t, max_steps=k)
        # GPU: its own CFL steps
        for dt_o in dts_o:
            dt = s.max_dt(Ud, prob.cfl)
            if dt > dt_o * (1 + 1e-9):  # clipped last step
                dt = dt_o
            max_ddt = max(max_ddt, abs(dt - dt_o) / dt_o)
            s.step(Ud, dt, 1)
        t += float(np.sum(dts_o))
        n += len(dts_o)
        hist.append((n, normwise_err(to_host(Ud), Uo)))
        print("step %d  t %.4f  normwise error %.3e  max rel dt difference %.2e" % (n, t, hist[-1][1], max_ddt),
              flush=True)
        if len(dts_o) < k:
            break
    assert s.status() == 0
    return n, hist, max_ddt


def test_four_quadrant_1024_to_t08(B):
    p = W.riemann2d(1024)
    n, hist, max_ddt = _run_both(B, p, p.t_end, 100000)
    assert n > 5000
    assert max_ddt <= 1e-11
    assert hist[-1][1] < TOL, hist


def test_viscous_cylinder_2048x1024_2000_steps(B):
    p = W.shock_cylinder()
    n, hist, max_ddt = _run_both(B, p, 1e9, p.n_steps)
    assert n == p.n_steps
    assert max_ddt <= 1e-11
    assert hist[-1][1] < TOL, hist
