"""A grid whose state holds more than 2^31 values: 32768 x 16640 cells, four planes of 5.45e8
cells = 2.18e9 doubles (about 115 GB of device memory with the solver's workspace), so that the
element offsets of the last plane's final rows only fit in 64-bit arithmetic.

The viscous periodic state is made with torch on the device (smooth, a few Fourier modes; no
output of the library is an input here).  One SSP-RK3 step with the grid's own CFL step (the
CFL reduction over all 5.45e8 cells, compared with the oracle's rate on the sampled patches: the
grid's step can only be smaller).  At sampled cells -- the first rows, the middle and the last
rows of the grid, where the offsets pass 2^31 -- the step equals the oracle's step of a 41 x 41
patch around the cell, on its central 17 x 17 cells (one step reaches 3 stages x 3 cells, so
cells 12 or more inside the patch do not see the patch's own boundary), within the 1e-10 bar."""
import numpy as np
import pytest

import oracle as O
from paper_2601_04400_gb300 import workloads as W
from jsutil import normwise_err, to_host

pytestmark = pytest.mark.gpu

NX, NY = 32768, 16640
PATCH, CORE = 41, 17
NEED_BYTES = 130 * 2 ** 30


def _state(torch, gamma):
    dx = 1.0 / NX
    Ly = NY * dx
    x = (torch.arange(NX, dtype=torch.float64, device="cuda") + 0.5) * dx
    y = (torch.arange(NY, dtype=torch.float64, device="cuda") + 0.5) * dx
    two_pi = 2.0 * np.pi

    def mode(kx, ky, ph):
        return torch.sin(two_pi * (kx * x[None, :] + ky * y[:, None] / Ly) + ph)

    U = torch.empty((4, NY, NX), dtype=torch.float64, device="cuda")
    rho = 1.0 + 0.2 * mode(3, 1, 0.3) + 0.05 * mode(40, 7, 1.1)
    u = 0.3 + 0.2 * mode(1, 2, 0.7)
    v = -0.2 + 0.15 * mode(2, 3, 2.1)
    p = 1.0 + 0.1 * mode(5, 4, 0.9) + 0.02 * mode(60, 30, 0.2)
    U[0] = rho
    U[1] = rho * u
    U[2] = rho * v
    U[3] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    del rho, u, v, p
    return U


def test_state_beyond_two_to_the_31_values_matches_oracle_patches():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < NEED_BYTES:
        pytest.skip("needs about 130 GB of free device memory")
    from paper_2601_04400_gb300 import binding as B
    assert 4 * NX * NY > 2 ** 31
    prob = W.Problem("maxsize", NX, NY, 0.0, 0.0, 1.0 / NX, 1.0 / NX, bc=(2, 2, 2, 2), mu=2e-6)
    s = B.Solver.from_problem(prob)
    U = _state(torch, prob.gamma)
    dt = s.max_dt(U, 0.5)
    cells = [(30, 25), (NX // 2, NY // 2), (NX - 25, NY - 30), (25, NY - 21), (NX - 21, 21)]
    h = PATCH // 2
    before = {}
    for (i, j) in cells:
        before[(i, j)] = to_host(U[:, j - h:j + h + 1, i - h:i + h + 1])
    s.step(U, dt, 1)
    assert s.status() == 0
    c0 = (PATCH - CORE) // 2
    for (i, j) in cells:
        Up = before[(i, j)]
        pp = W.Problem("patch", PATCH, PATCH, 0.0, 0.0, prob.dx, prob.dy, bc=(0, 0, 0, 0), mu=prob.mu)
        # the grid's CFL step bounds the patch's (a maximum over more cells)
        assert dt <= O.max_dt(pp, Up, 0.5) * (1.0 + 1e-15)
        ref = O.step(pp, Up, [dt])[:, c0:c0 + CORE, c0:c0 + CORE]
        got = to_host(U[:, j - h + c0:j - h + c0 + CORE, i - h + c0:i - h + c0 + CORE])
        assert normwise_err(got, ref) < 1e-10, (i, j, normwise_err(got, ref))
    # the last sampled rows lie where the offsets of plane 3 pass 2^31
    assert 3 * NX * NY + (NY - 30) * NX > 2 ** 31
    del U, s
    torch.cuda.empty_cache()
