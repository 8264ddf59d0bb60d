"""Parameter recovery through the differentiable solver (Sec. 3: the specific heat ratio
inferred from flow-field data by gradient descent, with Adam at a constant learning rate for
the Sod tube and a warm cosine-decay schedule for the shock-cylinder subdomain).

The loss is the multi-step objective of Sec. 2.4: the mean over the m unrolled steps of the
squared L2 distance between the predicted state U^{n+s} and the target state at that step,
optionally restricted to a subdomain (a cell mask).  Its gradient comes from the checkpointed
reverse pass of `autograd.rollout`, which injects each step's loss adjoint when the backward
pass reaches that step; gamma enters both the solver (parameter vector entry 0) and the
conserved initial state built from the primitive one (E = p / (gamma - 1) + rho |u|^2 / 2).
"""
import math

import torch

from . import autograd as A


class _PrimToCons(torch.autograd.Function):
    """U = prim_to_cons(W0) with the library's EOS kernel (js_prim_to_cons) at the solver's
    gamma; its derivative in gamma is analytic: only E = p/(gamma - 1) + rho |u|^2 / 2 depends
    on it, dE/dgamma = -p / (gamma - 1)^2.  W0 is data (no gradient)."""

    @staticmethod
    def forward(ctx, gamma, W0, solver):
        g = float(gamma)
        A._apply_theta(solver, torch.cat([gamma.detach().view(1).cpu(), A.theta_of(solver)[1:]]))
        ctx.save_for_backward(W0[3])
        ctx.g = g
        return solver.prim_to_cons(W0)

    @staticmethod
    def backward(ctx, U_bar):
        (p,) = ctx.saved_tensors
        dE = -p / (ctx.g - 1.0) ** 2
        return (U_bar[3] * dE).sum().to(torch.float64).cpu(), None, None


def prim_to_cons(solver, W0, gamma):
    """Conserved state [4, ny, nx] from primitive W0 = (rho, u, v, p) by the library kernel at
    gamma (which becomes the solver's gamma), differentiable in gamma."""
    return _PrimToCons.apply(gamma, W0, solver)


def multistep_loss(states, targets, mask=None):
    """(1/m) sum_s sum_cells sum_components (U_s - T_s)^2 over cells where mask is True.
    states, targets: [m, 4, ny, nx]; mask: bool [ny, nx] or None (every cell)."""
    d = states - targets
    if mask is not None:
        d = d * mask.to(d.dtype)
    return (d * d).sum() / states.shape[0]


def warm_cosine(k, warm, total, lr_start, lr_end):
    """Learning rate at iteration k: lr_start for the first `warm` iterations, then a cosine
    decay reaching lr_end at iteration `total` (and staying there)."""
    if k < warm:
        return lr_start
    if total <= warm:
        return lr_end
    x = min(1.0, (k - warm) / (total - warm))
    return lr_end + 0.5 * (lr_start - lr_end) * (1.0 + math.cos(math.pi * x))


def fit_gamma(solver, W0, targets, dts, gamma0, iters, lr=0.1, schedule=None, mask=None, outputs=None,
              checkpoint_every=None, betas=(0.9, 0.999)):
    """Recover gamma by Adam on the multi-step loss.

    solver: binding.Solver of the problem (its other parameters stay fixed); W0: primitive
    initial state, float64 CUDA tensor [4, ny, nx]; targets: [m, 4, ny, nx] states at the steps
    listed in `outputs` (default 1..m); dts: the fixed step sizes of the rollout (len(dts) >=
    max(outputs)); gamma0: initial guess; schedule: None (constant lr) or a function
    k -> learning rate; betas: Adam's moment decay rates.  Returns dict(gamma=[...], loss=[...]) with one entry per iteration
    (the loss and gamma before that iteration's update) and the final gamma last."""
    outputs = list(range(1, targets.shape[0] + 1)) if outputs is None else list(outputs)
    if len(outputs) != targets.shape[0] or max(outputs) > len(dts):
        raise ValueError("outputs must index one target per entry within the rollout")
    theta_rest = A.theta_of(solver)[1:].clone()
    g = torch.tensor(float(gamma0), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([g], lr=lr, betas=tuple(betas))
    hist = {"gamma": [], "loss": []}
    dts = list(dts)[:max(outputs)]
    for k in range(iters):
        if schedule is not None:
            for grp in opt.param_groups:
                grp["lr"] = schedule(k)
        opt.zero_grad()
        theta = torch.cat([g.view(1), theta_rest])
        U0 = prim_to_cons(solver, W0, g)
        states = A.rollout(solver, U0, theta, dts, outputs=outputs, checkpoint_every=checkpoint_every)
        loss = multistep_loss(states, targets, mask)
        loss.backward()
        hist["gamma"].append(g.item())
        hist["loss"].append(loss.item())
        opt.step()
        with torch.no_grad():
            g.clamp_(min=1.0 + 1e-6)  # gamma > 1 keeps the state physical
    hist["gamma"].append(g.item())
    solver.check()
    return hist
