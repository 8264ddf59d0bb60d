"""Degenerate inputs of the solver's entry points (GPU):

* grids below the WENO5 stencil's minimum (fewer than 6 cells along a used axis) and the 2^31-cell
  limit are refused with JS_ERR_ARG before anything is allocated;
* the smallest accepted grids (6 x 6 periodic, 6 x 6 four-quadrant with transmissive sides,
  6 x 1 Sod) take steps equal to the oracle's within the parity bar;
* zero steps (js_step, js_step_cfl, js_batch_step) leave the state bit for bit unchanged and
  report no error; negative step counts and a rollout of zero steps are JS_ERR_ARG."""
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


@pytest.mark.parametrize("nx,ny", [(5, 8), (8, 5), (8, 2), (2, 1)])
def test_grids_below_the_stencil_are_refused(B, nx, ny):
    p = W.random_periodic(8, 8, seed=0)
    with pytest.raises(B.JsError) as e:
        B.Solver(nx, ny, p.x0, p.y0, p.dx, p.dy, p.bc, p.gamma, p.mu, p.Pr, p.nu, p.inflow, 0, None, None)
    assert e.value.code == B.JS_ERR_ARG


def test_more_than_2_31_cells_are_refused(B):
    p = W.random_periodic(8, 8, seed=0)
    with pytest.raises(B.JsError) as e:
        B.Solver(65536, 32769, p.x0, p.y0, p.dx, p.dy, p.bc, p.gamma, p.mu, p.Pr, p.nu, p.inflow, 0, None, None)
    assert e.value.code == B.JS_ERR_ARG


@pytest.mark.parametrize("case", ["periodic", "quadrants", "sod"])
def test_smallest_grids_step_like_the_oracle(B, case):
    if case == "periodic":
        p = W.random_periodic(6, 6, seed=3, amp=0.1)
        U = O.prim_to_cons(p, p.W0)
    elif case == "quadrants":
        p = W.riemann2d(6)
        U = O.prim_to_cons(p, p.W0)
    else:
        p = W.sod(6)
        U = O.prim_to_cons(p, p.W0)
    dt = 0.4 * O.max_dt(p, U, 0.5)
    ref = O.step(p, U, [dt] * 3)
    s = B.Solver.from_problem(p)
    Ud = to_dev(U)
    s.step(Ud, dt, 3)
    assert s.status() == 0
    assert normwise_err(to_host(Ud), ref) < TOL


def test_zero_steps_change_nothing(B):
    import torch
    p = W.riemann2d(48, ny=40)
    U0 = to_dev(O.prim_to_cons(p, W.random_state(p, seed=1, amp=0.05)))
    s = B.Solver.from_problem(p)
    U = U0.clone()
    s.step(U, 1e-4, 0)
    t = torch.zeros((), dtype=torch.float64, device="cuda")
    s.step_cfl(U, 0.5, 0, t=t)
    assert s.status() == 0
    assert torch.equal(U, U0) and float(t) == 0.0
    with pytest.raises(B.JsError) as e:
        s.step(U, 1e-4, -1)
    assert e.value.code == B.JS_ERR_ARG
    with pytest.raises(B.JsError) as e:
        s.step_cfl(U, 0.5, -1)
    assert e.value.code == B.JS_ERR_ARG
    s.close()


def test_batched_zero_steps_and_empty_rollout(B):
    import torch
    probs = [W.riemann2d(48, ny=40), W.riemann2d(32, ny=24)]
    states = [to_dev(O.prim_to_cons(p, W.random_state(p, seed=4, amp=0.05))) for p in probs]
    b = B.Batch(probs)
    work = [U.clone() for U in states]
    b.set_states(work)
    b.step(0.5, 0)
    assert b.status() == 0
    for U, U0 in zip(work, states):
        assert torch.equal(U, U0)
    log = torch.zeros((0, len(probs)), dtype=torch.float64, device="cuda")
    with pytest.raises(B.JsError) as e:
        b.rollout_vjp(log, [torch.zeros_like(U) for U in states])
    assert e.value.code == B.JS_ERR_ARG
    with pytest.raises(B.JsError) as e:
        b.step(0.5, -1)
    assert e.value.code == B.JS_ERR_ARG
    b.close()
