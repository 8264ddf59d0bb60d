"""Training the neural flux through the solver (Sec. 2.3-2.4).

* The weight gradient of the multi-step window loss (checkpointed rollout, weights as an
  autograd input) equals the oracle's exact directional derivative (forward mode through
  the same steps) and central differences of the GPU loss.
* Block averaging (the downsampling of fine runs) equals numpy's block means.
* Adam training on block-averaged fine Sod runs lowers the window loss on fixed windows and
  makes the coarse solver closer to the fine one than the plain coarse solver (the
  qualitative result of Sec. 3, Fig. 4(c)-(f), on a reduced tube)."""
import numpy as np
import pytest

import oracle as O
from paper_2601_04400_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04400_gb300 import autograd as A
    from paper_2601_04400_gb300 import binding as B
    from paper_2601_04400_gb300 import inverse as I
    from paper_2601_04400_gb300 import neural as N
    B.lib()
    return torch, A, B, I, N


def test_block_average_equals_block_means(env):
    torch, A, B, I, N = env
    U = np.random.default_rng(0).standard_normal((4, 12, 18))
    got = B.block_average(torch.tensor(U, device="cuda"), 3, 2).cpu().numpy()
    ref = U.reshape(4, 6, 2, 6, 3).mean(axis=(2, 4))
    assert np.abs(got - ref).max() <= 1e-15 * np.abs(ref).max()


def test_window_loss_weight_gradient_matches_oracle(env):
    torch, A, B, I, N = env
    p = W.shock_cylinder(nx=48, ny=32, Lx=3.0, Ly=2.0, centre=(1.5, 1.0), radius=0.4, x_shock=0.7, viscous=False)
    U0 = O.prim_to_cons(p, p.W0)
    dt = 0.4 * O.max_dt(p, U0, 0.5)
    m = 4
    rng = np.random.default_rng(3)
    T = np.stack([O.step(p, U0, [dt] * (s + 1)) + 0.01 * rng.standard_normal(U0.shape) for s in range(m)])
    w = N.init_weights(5, zero_last=False).cpu().numpy() * 0.5
    norm = N.frame_norm(torch.tensor(U0), scale=0.2)
    dw = rng.standard_normal(w.size)
    # GPU: autograd through the checkpointed rollout
    s = B.Solver.from_problem(p)
    wt = torch.tensor(w, device="cuda", requires_grad=True)
    states = A.rollout(s, torch.tensor(U0, device="cuda"), A.theta_of(s), [dt] * m, outputs=list(range(1, m + 1)),
                       weights=wt, norm=norm, checkpoint_every=2)
    loss = I.multistep_loss(states, torch.tensor(T, device="cuda"))
    loss.backward()
    g_gpu = float(torch.dot(wt.grad, torch.tensor(dw, device="cuda")))
    # oracle: forward mode along dw
    g_ref, U, dU = 0.0, U0, np.zeros_like(U0)
    with O.neural(w, norm, dw=dw):
        for k in range(m):
            U, dU = O.step_tangent(p, U, dU, np.zeros(20), [dt])
            g_ref += 2.0 * np.sum((U - T[k]) * dU)
    g_ref /= m
    assert abs(g_gpu - g_ref) <= 1e-9 * abs(g_ref), (g_gpu, g_ref)
    # central differences of the GPU loss (h = 1e-7: larger steps cross ReLU kinks)
    h = 1e-7

    def L(e):
        with torch.no_grad():
            ws = torch.tensor(w + e * dw, device="cuda")
            st = A.rollout(s, torch.tensor(U0, device="cuda"), A.theta_of(s), [dt] * m, outputs=list(range(1, m + 1)),
                           weights=ws, norm=norm)
            return float(I.multistep_loss(st, torch.tensor(T, device="cuda")))
    fd = (L(h) - L(-h)) / (2 * h)
    assert abs(g_gpu - fd) <= 1e-5 * abs(fd), (g_gpu, fd)


def test_training_on_block_averaged_fine_sod_runs(env):
    torch, A, B, I, N = env
    nc, factor = 100, 2
    fine_p, coarse_p = W.sod(nc * factor), W.sod(nc)
    fine = B.Solver.from_problem(fine_p)
    Uf = fine.prim_to_cons(torch.tensor(fine_p.W0, device="cuda"))
    coarse = B.Solver.from_problem(coarse_p)
    dt = 0.4 * coarse_p.dx / 1.2
    T = N.make_targets(fine, Uf, dt, 60, factor)
    tr = N.Trainer(coarse, T, dt, N.frame_norm(T, scale=0.1), unroll=8, lr=1e-3, seed=0)
    windows = [0, 13, 26, 39, 52]
    with torch.no_grad():
        before = [float(tr.window_loss(k, tr.w)) for k in windows]
    base = tr.rollout_error(0, 60, neural=False)
    rng = np.random.default_rng(0)
    for _ in range(100):
        tr.step(int(rng.integers(0, 53)))
    with torch.no_grad():
        after = [float(tr.window_loss(k, tr.w)) for k in windows]
    assert sum(after) < 0.7 * sum(before), (before, after)
    assert tr.rollout_error(0, 60, neural=True) < base
