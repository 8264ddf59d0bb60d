"""Differentiable rollouts of the SSP-RK3 solver step (Sec. 2: U^{n+k} = S(U^{n+k-1}, theta),
gradients by the chain rule through the unrolled steps, Fig. 1(d)).

Forward steps run js_step; the backward pass walks the steps in reverse.  Only every
`checkpoint_every`-th state is kept (default ceil(sqrt(n))); during the backward pass each
segment is re-run from its checkpoint with js_step_taped (which records the stage states of
every step) and reversed with js_step_vjp_taped, so a rollout of n steps holds about
sqrt(n) checkpoints plus 3 sqrt(n) stage states instead of n states.  On 2D grids the tape
also records the WENO5 internals of every stage (about 1.3 KB per cell and step) when they
fit in half of the free device memory, which spares the reverse pass their recompute.

theta is the 20-entry parameter vector of the library (gamma, mu, Pr, nu, then the inflow
state rho, u, v, p of the x-low, x-high, y-low and y-high sides); its gradient is returned
for gamma, for mu and Pr when mu > 0, for nu when nu > 0 and for the inflow states of inflow
sides (the other entries receive zero).

With `weights` (the 6388 parameters of the neural flux of Sec. 2.3) the steps include the
neural flux and the backward pass also returns the weights' gradient (the per-step chain
rule of Sec. 2.4 through every unrolled step).
"""
import math

import torch

from . import binding as B


def theta_of(solver):
    """Current parameter vector of a Solver as a float64 CPU tensor."""
    sp = solver._spec
    t = torch.zeros(B.JS_NPARAM, dtype=torch.float64)
    t[0], t[1], t[2], t[3] = sp["gamma"], sp["mu"], sp["Pr"], sp["nu"]
    t[4:] = torch.as_tensor(sp["inflow"].reshape(16))
    return t


def _apply_theta(solver, theta):
    th = theta.detach().to("cpu", torch.float64)
    solver.set_params(gamma=float(th[0]), mu=float(th[1]), Pr=float(th[2]), nu=float(th[3]),
                      inflow=th[4:].numpy().reshape(4, 4))


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, theta, weights, solver, dts, outputs, every, internals, nn_cfg):
        _apply_theta(solver, theta)
        ctx.nn = None
        if weights is not None:
            # a private copy: the library reads the parameters at every stage, also when the
            # backward pass re-runs the segments
            w = weights.detach().to(U0.device, torch.float64).contiguous().clone()
            solver.set_neural(w, nn_cfg["norm"], fp32=nn_cfg.get("fp32", False))
            ctx.nn = (w, nn_cfg)
        n = len(dts)
        want = {k: i for i, k in enumerate(outputs)}
        U = U0.detach().clone().contiguous()
        ckpts = []
        outs = [None] * len(outputs)
        if 0 in want:
            outs[want[0]] = U.clone()
        for k in range(n):
            if k % every == 0:
                ckpts.append(U.clone())
            solver.step(U, dts[k], 1)
            if k + 1 in want:
                outs[want[k + 1]] = U.clone()
        ctx.solver, ctx.dts, ctx.outputs, ctx.every = solver, list(dts), list(outputs), every
        ctx.internals = internals
        ctx.w_device = None if weights is None else weights.device
        ctx.ckpts = ckpts
        ctx.theta = theta.detach().clone()
        return torch.stack(outs)

    @staticmethod
    def backward(ctx, g):
        solver, dts, every = ctx.solver, ctx.dts, ctx.every
        _apply_theta(solver, ctx.theta)
        n = len(dts)
        inject = {}
        for i, k in enumerate(ctx.outputs):
            inject[k] = g[i] if k not in inject else inject[k] + g[i]
        lam = torch.zeros_like(g[0])
        if n in inject:
            lam += inject[n]
        pbar = torch.zeros(B.JS_NPARAM, dtype=torch.float64, device=g.device)
        wbar = None
        if ctx.nn is not None:
            w, cfg = ctx.nn
            wbar = torch.zeros_like(w)
            solver.set_neural(w, cfg["norm"], w_bar=wbar, fp32=cfg.get("fp32", False))
        scratch = torch.empty_like(lam)
        weno = ctx.internals
        if weno is None:
            free = torch.cuda.mem_get_info(g.device)[0]
            weno = solver.tape_weno_bytes(every) < 0.5 * free
        solver.tape_reserve(every, weno=bool(weno))
        for seg in reversed(range(len(ctx.ckpts))):
            start = seg * every
            stop = min(start + every, n)
            # re-run the segment, recording every step's stage states on the tape
            U = ctx.ckpts[seg].clone()
            for k in range(start, stop):
                solver.step_taped(U, dts[k], k - start)
            for k in reversed(range(start, stop)):
                solver.step_vjp_taped(k - start, dts[k], lam, lam_n=scratch, p_bar=pbar)
                lam, scratch = scratch, lam
                if k in inject:
                    lam = lam + inject[k]
        st = solver.status()
        if ctx.nn is not None:
            solver.set_neural(ctx.nn[0], ctx.nn[1]["norm"], fp32=ctx.nn[1].get("fp32", False))
        if st != 0:
            raise B.JsError(st, "rollout backward")
        gw = None if wbar is None else wbar.to(ctx.w_device)
        return lam, pbar.to(ctx.theta.device), gw, None, None, None, None, None, None


def rollout(solver, U0, theta, dts, outputs=None, checkpoint_every=None, tape_internals=None, weights=None,
            norm=None, fp32=False):
    """Differentiable rollout.

    solver: binding.Solver; U0: float64 CUDA tensor [4, ny, nx]; theta: float64 tensor [20]
    (see module docstring); dts: list of step sizes (one per step).  outputs: step indices
    whose states are returned stacked (default: only the final state, index len(dts)).
    tape_internals: record the WENO5 internals on the tape (True / False; None decides by
    free device memory).  The gradient is the same either way.
    weights: float64 tensor [6388] of neural-flux parameters (Sec. 2.3) or None; norm: its
    input normalisation and output scale (mean[4], sd[4], scale[4]); fp32: FP32 network
    arithmetic.  The solver keeps the neural flux switched on after the call.
    Returns a tensor [len(outputs), 4, ny, nx] (or [4, ny, nx] for the default)."""
    n = len(dts)
    default = outputs is None
    outputs = [n] if default else list(outputs)
    every = checkpoint_every or max(1, int(math.ceil(math.sqrt(max(n, 1)))))
    if weights is not None and norm is None:
        raise ValueError("the neural flux needs its normalisation (norm)")
    cfg = None if weights is None else {"norm": norm, "fp32": bool(fp32)}
    out = _Rollout.apply(U0, theta, weights, solver, list(dts), outputs, every, tape_internals, cfg)
    return out[0] if default else out
