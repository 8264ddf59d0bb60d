"""Training the neural flux of Sec. 2.3 on coarse grids against block-averaged fine runs
(Sec. 2.4).

* Targets: a fine run whose grid is `factor` times finer in every direction takes `factor`
  steps of dt/factor per coarse step (the same CFL number); after each coarse step its state
  is block-averaged (js_block_average) onto the coarse grid.
* Loss: the multi-step objective of Sec. 2.4 over windows of m unrolled coarse steps started
  from a target state, (1/m) sum_s ||U^{n+s} - T^{n+s}||^2, its gradient with respect to the
  6388 network parameters from the checkpointed reverse pass (autograd.rollout).
* Optimiser: Adam (the paper trains with Adam at a constant learning rate of 1e-3).

The network starts with its last layer at zero, i.e. as the plain solver, so the training
loss starts at the coarse solver's own error.
"""
import math

import numpy as np
import torch

from . import autograd as A
from . import binding as B
from . import inverse as I

NPARAM = B.JS_NN_NPARAM
LAYERS = ((4, 16, 0), (16, 32, 592), (32, 4, 5232))  # (in, out, offset) of each 3x3 layer


def init_weights(seed=0, zero_last=True, device="cuda"):
    """He-uniform weights for the ReLU layers, zero biases; the tanh layer zero when
    zero_last (the network then adds nothing until trained)."""
    g = torch.Generator().manual_seed(int(seed))
    w = torch.zeros(NPARAM, dtype=torch.float64)
    for k, (cin, cout, off) in enumerate(LAYERS):
        n = cout * cin * 9
        if k == len(LAYERS) - 1 and zero_last:
            continue
        bound = math.sqrt(6.0 / (cin * 9))
        w[off:off + n] = (torch.rand(n, generator=g, dtype=torch.float64) * 2.0 - 1.0) * bound
    return w.to(device)


def frame_norm(states, scale=0.1):
    """Normalisation of the network input from states [..., 4, ny, nx]: mean and standard
    deviation of rho and E, and of both momentum components pooled (normal and tangential
    momentum then share them, mean zero); output scale = scale x those deviations."""
    s = states.reshape(-1, 4, states.shape[-2], states.shape[-1]).double()
    r, mx, my, E = s[:, 0], s[:, 1], s[:, 2], s[:, 3]
    m = torch.cat([mx.reshape(-1), my.reshape(-1)])
    sd = [float(r.std()) + 1e-6, float(m.std()) + 1e-6, float(m.std()) + 1e-6, float(E.std()) + 1e-6]
    mean = [float(r.mean()), 0.0, 0.0, float(E.mean())]
    return np.array(mean + sd + [scale * v for v in sd])


def make_targets(fine, U_fine, dt, steps, factor):
    """Coarse-grid targets [steps + 1, 4, ny/f, nx/f] (index 0: the block-averaged initial
    state): `fine` (a Solver) advances U_fine (float64 CUDA, modified) by `factor` steps of
    dt/factor per coarse step.  1D grids (ny == 1) average along x only."""
    fy = factor if U_fine.shape[1] > 1 else 1
    out = [B.block_average(U_fine, factor, fy)]
    for _ in range(steps):
        fine.step(U_fine, dt / factor, factor)
        out.append(B.block_average(U_fine, factor, fy))
    fine.check()
    return torch.stack(out)


class Trainer:
    """Adam on the network parameters over windows of `unroll` coarse steps."""

    def __init__(self, coarse, targets, dt, norm, weights=None, unroll=8, lr=1e-3, fp32=False, seed=0):
        self.solver = coarse
        self.targets = targets
        self.dt = float(dt)
        self.norm = np.asarray(norm, dtype=np.float64)
        self.m = int(unroll)
        self.fp32 = bool(fp32)
        w = init_weights(seed, device=targets.device) if weights is None else weights.detach().clone()
        self.w = torch.nn.Parameter(w)
        self.opt = torch.optim.Adam([self.w], lr=lr)
        self.theta = A.theta_of(coarse)

    def window_loss(self, start, weights):
        """Multi-step loss of the window starting at target `start`."""
        m = self.m
        states = A.rollout(self.solver, self.targets[start].contiguous(), self.theta, [self.dt] * m,
                           outputs=list(range(1, m + 1)), weights=weights, norm=self.norm, fp32=self.fp32)
        return I.multistep_loss(states, self.targets[start + 1:start + m + 1])

    def step(self, start):
        """One Adam iteration on the window starting at `start`; returns its loss (before)."""
        self.opt.zero_grad()
        loss = self.window_loss(start, self.w)
        loss.backward()
        self.opt.step()
        return loss.item()

    def rollout_error(self, start, n, neural=True):
        """Mean over n coarse steps from target `start` of ||U^s - T^s||^2, with the network
        (neural) or as the plain coarse solver."""
        U = self.targets[start].clone().contiguous()
        if neural:
            self.solver.set_neural(self.w.detach().contiguous(), self.norm, fp32=self.fp32)
        else:
            self.solver.set_neural(None)
        err = 0.0
        for s in range(1, n + 1):
            self.solver.step(U, self.dt, 1)
            err += float(((U - self.targets[start + s]) ** 2).sum())
        self.solver.check()
        return err / n
