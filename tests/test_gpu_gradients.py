"""End-to-end gradients of a shock-cylinder rollout (the adjoint workload: 64^2 x 16 steps, and
the full configuration, 512^2 x 400 steps with sqrt(N) checkpointing):
loss = sum over fluid cells of (rho - rho_target)^2 dx dy after n steps, the target being a
run at Mach 2.2; gradients with respect to the shock Mach number (initial condition and
inflow state), gamma and mu from the checkpointed reverse pass, against central finite
differences (h = 1e-6) of the GPU forward solver, and checkpointing that does not change
the gradient.

At full size the gradients also equal the exact discrete derivatives, the oracle's forward
mode stored in tests/golden/adjoint_case_512_gradients.txt, to 1e-9.  There the loss is not
smooth in mu at the 1e-6 level (branches of the scheme switch within the difference stencil):
central differences in mu for h from 5e-7 to 8e-6 all sit about 2e-6 (relative) from the
exact derivative, so the finite-difference bound for mu at that size is 5e-6."""
import numpy as np
import pytest

from conftest import golden
from paper_2601_04400_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N, STEPS, MU0 = 64, 16, 3.9443e-3


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04400_gb300 import autograd as A
    from paper_2601_04400_gb300 import binding as B
    B.lib()
    return torch, B, A


def _problem(M, gamma=1.4, mu=MU0, n=N, steps=STEPS):
    p = W.adjoint_case(n, mach=M, gamma=gamma, n_steps=steps)
    return p.with_(mu=mu)


def _cons(W0, gamma):
    r, u, v, p = W0
    return np.stack([r, r * u, r * v, p / (gamma - 1.0) + 0.5 * r * (u * u + v * v)])


def _setup(torch, B, n, steps):
    # fixed dt from CFL 0.5 on the Mach-2.2 initial state, used by every run
    pt = _problem(2.2, n=n, steps=steps)
    s = B.Solver.from_problem(pt)
    Ut = torch.tensor(_cons(pt.W0, pt.gamma), device="cuda")
    dt = s.max_dt(Ut, 0.5)
    s.step(Ut, dt, steps)
    _, tag = s.ib_info()
    fluid = torch.tensor(tag == 0, device="cuda")
    return dt, Ut[0].clone(), fluid


def _loss_fd(torch, B, dt, rho_t, fluid, M, gamma, mu, n, steps):
    p = _problem(M, gamma, mu, n, steps)
    s = B.Solver.from_problem(p)
    U = torch.tensor(_cons(p.W0, gamma), device="cuda")
    s.step(U, dt, steps)
    d = (U[0] - rho_t) * fluid
    return float((d * d).sum()) * p.dx * p.dy


@pytest.mark.parametrize("n,steps", [(N, STEPS), (512, 400)])
def test_rollout_gradients_match_central_differences(env, n, steps):
    torch, B, A = env
    dt, rho_t, fluid = _setup(torch, B, n, steps)
    M, gamma, mu = 2.0, 1.4, MU0
    p = _problem(M, gamma, mu, n, steps)
    s = B.Solver.from_problem(p)
    U0 = torch.tensor(_cons(p.W0, gamma), device="cuda", requires_grad=True)
    theta = A.theta_of(s).requires_grad_(True)
    UN = A.rollout(s, U0, theta, [dt] * steps)  # checkpoints every ceil(sqrt(steps)) steps
    d = (UN[0] - rho_t) * fluid
    loss = (d * d).sum() * p.dx * p.dy
    loss.backward()
    lam0 = U0.grad.detach().cpu().numpy()
    pb = theta.grad.detach().cpu().numpy()
    # chain rule through the initial condition and the inflow state
    W0 = p.W0
    dWdM, dWdg = W.post_shock_state_derivs(M, 1.0, 1.0, gamma)
    behind = (W.cell_centres(p.nx, p.ny, 0, 0, p.dx, p.dy)[0] < p.meta["x_shock"])
    r, u, v, pr = W0
    Jc = lambda dW: np.stack([dW[0], dW[0] * u + r * dW[1], dW[0] * v + r * dW[2],
                              dW[0] * 0.5 * (u * u + v * v) + r * (u * dW[1] + v * dW[2]) + dW[3] / (gamma - 1.0)])
    dU_dM = Jc(np.where(behind, 1.0, 0.0)[None] * np.asarray(dWdM)[:, None, None])
    dU_dg = Jc(np.where(behind, 1.0, 0.0)[None] * np.asarray(dWdg)[:, None, None])
    dU_dg[3] += -pr / (gamma - 1.0) ** 2
    g_M = np.sum(lam0 * dU_dM) + np.dot(pb[4:8], dWdM)
    g_g = np.sum(lam0 * dU_dg) + pb[0] + np.dot(pb[4:8], dWdg)
    g_mu = pb[1]
    h = 1e-6
    fd = lambda f: (f(h) - f(-h)) / (2 * h)
    fd_M = fd(lambda e: _loss_fd(torch, B, dt, rho_t, fluid, M + e, gamma, mu, n, steps))
    fd_g = fd(lambda e: _loss_fd(torch, B, dt, rho_t, fluid, M, gamma + e, mu, n, steps))
    fd_mu = fd(lambda e: _loss_fd(torch, B, dt, rho_t, fluid, M, gamma, mu + e, n, steps))
    fd_tol = (1e-6, 1e-6, 1e-6 if n < 512 else 5e-6)
    for got, ref, tol in zip((g_M, g_g, g_mu), (fd_M, fd_g, fd_mu), fd_tol):
        assert abs(got - ref) <= tol * abs(ref), (got, ref)
    if n == 512:
        dt_o, L_o, dM, dg, dmu = golden("adjoint_case_512_gradients.txt")[0]
        assert dt == dt_o  # the GPU's CFL step equals the oracle's bit for bit
        for got, ref in ((g_M, dM), (g_g, dg), (g_mu, dmu)):
            assert abs(got - ref) <= 1e-9 * abs(ref), (got, ref)


def test_checkpointing_does_not_change_the_gradient(env):
    torch, B, A = env
    p = _problem(2.0)
    s = B.Solver.from_problem(p)
    U0 = torch.tensor(_cons(p.W0, p.gamma), device="cuda")
    dt = 0.5 * s.max_dt(U0, 0.5)
    grads = []
    # segment lengths 1, 3, 12, each with and without the WENO internals on the tape
    for every, internals in ((1, False), (3, True), (3, False), (12, True)):
        U = U0.clone().requires_grad_(True)
        th = A.theta_of(s).requires_grad_(True)
        out = A.rollout(s, U, th, [dt] * 12, outputs=[4, 12], checkpoint_every=every,
                        tape_internals=internals)
        (out[0, 0].square().sum() + out[1, 3].sum()).backward()
        grads.append((U.grad.cpu().numpy(), th.grad.numpy()))
    for gU, gp in grads[1:]:
        assert np.abs(gU - grads[0][0]).max() <= 1e-12 * np.abs(grads[0][0]).max()
        assert np.abs(gp - grads[0][1]).max() <= 1e-12 * np.abs(grads[0][1]).max()
