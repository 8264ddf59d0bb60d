"""js_max_dt_noalloc -- the CFL time step for callers that cannot allocate device memory
(for example a host application that owns every device allocation through its own pool) --
returns what the context-based js_max_dt returns, bit for bit, and rejects the same
non-physical states.  Its scratch is a file-scope device array
shared by all calls, so two calls in a row must not see each other's partial results.
Collected last, so that a run stopping at the first failure has run every other test."""
import numpy as np
import pytest

from paper_2601_04400_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04400_gb300 import binding as B
    B.lib()
    return torch, B


def _case(torch, B, prob, seed):
    s = B.Solver.from_problem(prob)
    W0 = torch.tensor(W.random_state(prob, seed=seed, amp=0.05), dtype=torch.float64, device="cuda")
    U1 = s.prim_to_cons(W0)
    U2 = U1.clone()
    s.step(U2, 0.5 * s.max_dt(U2, prob.cfl), 3)
    n, tag = s.ib_info()
    tag_dev = torch.tensor(tag, dtype=torch.uint8, device="cuda") if n > 0 else None
    g, p, _ = B.make_structs(prob.nx, prob.ny, prob.x0, prob.y0, prob.dx, prob.dy, prob.bc, prob.gamma, prob.mu,
                             prob.Pr, prob.nu, prob.inflow, prob.wall)
    return s, (U1, U2), tag_dev, g, p


def test_noalloc_cfl_matches_js_max_dt_on_consecutive_calls():
    torch, B = _setup()
    # the larger grid first: the smaller one must not pick up its leftover partials
    for prob, seed in ((W.shock_cylinder(nx=512, ny=256), 1), (W.riemann2d(96, ny=80), 2)):
        s, states, tag_dev, g, p = _case(torch, B, prob, seed)
        got = []
        for U in states:
            ref = s.max_dt(U, prob.cfl)
            dt = B.js_max_dt_noalloc(g, p, U, tag_dev, prob.cfl)
            assert dt == ref
            got.append(dt)
        assert got[0] != got[1]  # the two calls reduced different states
        s.close()


def test_noalloc_cfl_rejects_grids_beyond_the_static_scratch():
    torch, B = _setup()
    U = torch.ones((4, 8, 8), dtype=torch.float64, device="cuda")
    g, p, _ = B.make_structs(4096, 2049, 0.0, 0.0, 1.0, 1.0, (0, 0, 0, 0), 1.4, 0.0, 0.72, 0.0,
                             np.tile([1.0, 0.0, 0.0, 1.0], (4, 1)))
    with pytest.raises(B.JsError) as e:
        B.js_max_dt_noalloc(g, p, U, None, 0.5)
    assert e.value.code == B.JS_ERR_ARG


def test_noalloc_cfl_rejects_non_physical_states_like_js_max_dt():
    torch, B = _setup()
    prob = W.shock_cylinder(nx=256, ny=128)
    s, (U1, _), tag_dev, g, p = _case(torch, B, prob, 3)
    n, tag = s.ib_info()
    j, i = np.argwhere(tag == 0)[1234]
    for bad in (-0.25, float("nan")):
        U = U1.clone()
        U[0, j, i] = bad
        codes = []
        for call in (lambda: s.max_dt(U, prob.cfl), lambda: B.js_max_dt_noalloc(g, p, U, tag_dev, prob.cfl)):
            with pytest.raises(B.JsError) as e:
                call()
            codes.append(e.value.code)
        assert codes == [B.JS_ERR_NONPHYSICAL] * 2
    # after the rejected calls the shared scratch still gives the right answer
    assert B.js_max_dt_noalloc(g, p, U1, tag_dev, prob.cfl) == s.max_dt(U1, prob.cfl)
    s.close()
