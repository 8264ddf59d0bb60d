"""Multi-step unrolled loss (Sec. 2.4) and gamma recovery (Sec. 3) through the CUDA path.

The gradient of L = (1/m) sum_s ||U^s - T^s||^2 (over a subdomain in 2D) with respect to gamma
-- entering the solver and the conserved initial state -- from the checkpointed reverse pass,
against the oracle's exact discrete derivative (forward-mode dual numbers through the same
steps) and against central finite differences of the GPU forward solver.  Targets are
oracle runs at a known gamma (1.4 for Sod, 2 for the cylinder subdomain, whose recovery
starts from 1.4 as in the paper's)."""
import numpy as np
import pytest

import oracle as O
from paper_2601_04400_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GAMMA_TRUE = 1.4


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04400_gb300 import binding as B
    from paper_2601_04400_gb300 import inverse as I
    B.lib()
    return torch, B, I


def _cons(W0, gamma):
    r, u, v, p = W0
    return np.stack([r, r * u, r * v, p / (gamma - 1.0) + 0.5 * r * (u * u + v * v)])


def _targets(prob, dts, outputs, gamma):
    th = O.theta_of(prob.with_(gamma=gamma))
    U, k, out = _cons(prob.W0, gamma), 0, []
    for s in outputs:
        U = O.step(prob, U, dts[k:s], theta=th)
        k = s
        out.append(U.copy())
    return np.stack(out)


def _oracle_grad(prob, dts, outputs, T, gamma, mask):
    """dL/dgamma by forward mode through the oracle."""
    th = O.theta_of(prob.with_(gamma=gamma))
    dth = np.zeros_like(th)
    dth[0] = 1.0
    U = _cons(prob.W0, gamma)
    dU = np.zeros_like(U)
    dU[3] = -prob.W0[3] / (gamma - 1.0) ** 2
    k, g = 0, 0.0
    for i, s in enumerate(outputs):
        U, dU = O.step_tangent(prob, U, dU, dth, dts[k:s], theta=th)
        k = s
        g += 2.0 * np.sum(((U - T[i]) * dU)[:, mask])
    return g / len(outputs)


def _cases():
    sod = W.sod(200, t_end=0.05)
    U0 = _cons(sod.W0, GAMMA_TRUE)
    _, dts = O.run_to(sod, U0, 0.5, 0.05)
    yield "sod200", sod, list(dts), list(range(3, len(dts) + 1, 3)), np.ones((1, 200), bool)
    cyl = W.shock_cylinder(nx=96, ny=64, Lx=6.0, Ly=4.0, centre=(2.0, 2.0), x_shock=1.0, Re=1000.0, n_steps=12)
    dt = O.max_dt(cyl, _cons(cyl.W0, GAMMA_TRUE), 0.5)
    X, Y = W.cell_centres(cyl.nx, cyl.ny, cyl.x0, cyl.y0, cyl.dx, cyl.dy)
    yield "cylinder96x64_subdomain", cyl, [dt] * 12, [4, 8, 12], (X <= 1.5) & (Y <= 1.0)


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_multistep_loss_gradient(env, case):
    torch, B, I = env
    from paper_2601_04400_gb300 import autograd as A
    _, prob, dts, outputs, mask = case
    T = _targets(prob, dts, outputs, GAMMA_TRUE)
    gamma = 1.5
    s = B.Solver.from_problem(prob.with_(gamma=gamma))
    W0 = torch.tensor(prob.W0, device="cuda")
    Td = torch.tensor(T, device="cuda")
    md = torch.tensor(mask, device="cuda")

    def loss_at(gm, grad):
        g = torch.tensor(gm, dtype=torch.float64, requires_grad=grad)
        theta = A.theta_of(s)
        theta = torch.cat([g.view(1), theta[1:]])
        states = A.rollout(s, I.prim_to_cons(s, W0, g), theta, dts[:outputs[-1]], outputs=outputs)
        L = I.multistep_loss(states, Td, md)
        if grad:
            L.backward()
            return L.item(), g.grad.item()
        return L.item(), None

    _, g_gpu = loss_at(gamma, True)
    g_ref = _oracle_grad(prob, dts, outputs, T, gamma, mask)
    assert abs(g_gpu - g_ref) <= 1e-9 * abs(g_ref), (g_gpu, g_ref)
    h = 1e-6
    fd = (loss_at(gamma + h, False)[0] - loss_at(gamma - h, False)[0]) / (2 * h)
    assert abs(g_gpu - fd) <= 1e-6 * abs(fd), (g_gpu, fd)
    assert s.status() == 0


def test_gamma_recovery_sod_constant_learning_rate(env):
    """Adam at the constant learning rate 0.1 (as for the Sod tube of Sec. 3), from 2.0."""
    torch, B, I = env
    prob = W.sod(200, t_end=0.1)
    _, dts = O.run_to(prob, _cons(prob.W0, GAMMA_TRUE), 0.5, 0.1)
    outputs = list(range(4, len(dts) + 1, 4))
    T = torch.tensor(_targets(prob, list(dts), outputs, GAMMA_TRUE), device="cuda")
    s = B.Solver.from_problem(prob.with_(gamma=2.0))
    h = I.fit_gamma(s, torch.tensor(prob.W0, device="cuda"), T, list(dts), 2.0, iters=60, lr=0.1, outputs=outputs)
    loss = np.array(h["loss"])
    assert loss[-10:].min() < 1e-3 * loss[0]
    assert abs(h["gamma"][-1] - GAMMA_TRUE) < 0.03


def test_gamma_recovery_cylinder_subdomain_warm_cosine(env):
    """Loss restricted to the subdomain [0, 1.5] x [0, 1]; constant learning rate, then a
    cosine decay (the schedule of the shock-cylinder recovery of Sec. 3); as in the paper's
    recovery, the initial guess is 1.4 and the target data are made with gamma = 2."""
    torch, B, I = env
    prob = W.shock_cylinder(nx=96, ny=64, Lx=6.0, Ly=4.0, centre=(2.0, 2.0), x_shock=1.0, Re=1000.0, n_steps=40)
    dt = O.max_dt(prob, _cons(prob.W0, GAMMA_TRUE), 0.5)
    dts = [dt] * 40
    outputs = list(range(4, 41, 4))
    T = torch.tensor(_targets(prob, dts, outputs, 2.0), device="cuda")
    X, Y = W.cell_centres(prob.nx, prob.ny, prob.x0, prob.y0, prob.dx, prob.dy)
    mask = torch.tensor((X <= 1.5) & (Y <= 1.0), device="cuda")
    s = B.Solver.from_problem(prob.with_(gamma=1.4))
    # a short second-moment memory: Adam's default 0.999 remembers the large early gradients
    # and stalls past the overshoot
    h = I.fit_gamma(s, torch.tensor(prob.W0, device="cuda"), T, dts, 1.4, iters=80, lr=0.05, mask=mask,
                    outputs=outputs, betas=(0.9, 0.9), schedule=lambda k: I.warm_cosine(k, 30, 80, 0.05, 5e-4))
    assert abs(h["gamma"][-1] - 2.0) < 5e-3
    assert h["loss"][-1] < 1e-4 * h["loss"][0]


def test_initial_state_depends_on_gamma_through_the_energy_only(env):
    """U0 = js_prim_to_cons(W0) at gamma; dU0/dgamma is -p/(gamma-1)^2 in the energy, 0 elsewhere."""
    torch, B, I = env
    p = W.riemann2d(24, ny=16).with_(gamma=1.4)
    s = B.Solver.from_problem(p)
    W0 = torch.tensor(np.random.default_rng(1).uniform(0.5, 2.0, (4, 16, 24)), device="cuda")
    g = torch.tensor(1.4, dtype=torch.float64, requires_grad=True)
    U = I.prim_to_cons(s, W0, g)
    r, u, v, pr = W0
    assert torch.allclose(U[3], pr / 0.4 + 0.5 * r * (u * u + v * v), rtol=1e-15, atol=0)
    (dg,) = torch.autograd.grad(U[3].sum(), g, retain_graph=True)
    assert float(dg) == pytest.approx(float((-pr / 0.4 ** 2).sum()), rel=1e-14)
    (d0,) = torch.autograd.grad(U[:3].sum(), g, allow_unused=True)
    assert d0 is None or float(d0) == 0.0
    g2 = torch.tensor(1.6, dtype=torch.float64, requires_grad=True)
    U2 = I.prim_to_cons(s, W0, g2)
    assert torch.allclose(U2[3], pr / 0.6 + 0.5 * r * (u * u + v * v), rtol=1e-15, atol=0)
    assert s._spec["gamma"] == 1.6
    s.close()
