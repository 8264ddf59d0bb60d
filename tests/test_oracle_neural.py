"""Pins of the oracle's neural flux (Sec. 2.3): the three-layer network against torch's own
convolution, the wiring of the face images into the flux (rebuilt independently from the
oracle's pinned WENO5 and torch's conv2d), the zero network, the transpose symmetry and the
weight tangent against finite differences."""
import numpy as np
import pytest

import oracle as O
from paper_2601_04400_gb300 import workloads as W

torch = pytest.importorskip("torch")
import torch.nn.functional as F  # noqa: E402

NP = 6388


def _params(seed, amp=0.15):
    return np.random.default_rng(seed).standard_normal(NP) * amp


def _norm(scale=0.3):
    # frame channels (rho, normal momentum, tangential momentum, E)
    return np.concatenate([[1.0, 0.1, 0.05, 2.5], [0.3, 0.4, 0.4, 0.8], np.full(4, scale)])


def _torch_net(w, X, scale):
    t = torch.tensor(w)
    w1, b1 = t[:576].view(16, 4, 3, 3), t[576:592]
    w2, b2 = t[592:5200].view(32, 16, 3, 3), t[5200:5232]
    w3, b3 = t[5232:6384].view(4, 32, 3, 3), t[6384:]
    x = torch.tensor(X)[None]
    y = F.conv2d(torch.relu(F.conv2d(torch.relu(F.conv2d(x, w1, b1, padding=1)), w2, b2, padding=1)), w3, b3,
                 padding=1)
    return (torch.tensor(scale)[:, None, None] * torch.tanh(y[0])).numpy()


def test_parameter_count_is_the_papers():
    assert O.nn_nparam() == NP  # 4*16*9+16 + 16*32*9+32 + 32*4*9+4


@pytest.mark.parametrize("shape", [(5, 7), (1, 9), (12, 3)])
def test_network_equals_torch_convolutions(shape):
    w = _params(1)
    X = np.random.default_rng(2).standard_normal((4,) + shape)
    with O.neural(w, _norm(0.7)):
        Y = O.nn_eval(X)
    ref = _torch_net(w, X, np.full(4, 0.7))
    assert np.abs(Y - ref).max() <= 1e-13 * np.abs(ref).max()


def test_zero_network_leaves_the_solver_unchanged():
    p = W.random_periodic(14, 11, seed=3, mu=2e-3)
    U = O.prim_to_cons(p, p.W0)
    ref = O.step(p, U, [2e-3] * 2)
    with O.neural(np.zeros(NP), _norm()):
        got = O.step(p, U, [2e-3] * 2)
    assert np.array_equal(got, ref)


def _faces_prim(Wp, nx, ny):
    """WENO5 face states (left-biased from the cell below/left, right-biased from the cell
    above/right) of a periodic primitive field, from the oracle's pinned scalar WENO5."""
    def states(q, axis):
        n = q.shape[axis]
        qL = np.zeros(q.shape[:axis] + (n + 1,) + q.shape[axis + 1:])
        qR = np.zeros_like(qL)
        for f in range(n + 1):
            a, b = f - 1, f  # cells left / right of face f (periodic)
            take = lambda k: np.take(q, k % n, axis=axis)
            st = np.stack([take(a - 2), take(a - 1), take(a), take(a + 1), take(a + 2)], -1)
            sr = np.stack([take(b + 2), take(b + 1), take(b), take(b - 1), take(b - 2)], -1)
            idx = [slice(None)] * q.ndim
            idx[axis] = f
            qL[tuple(idx)] = np.apply_along_axis(lambda v: O.weno5(v), -1, st)
            qR[tuple(idx)] = np.apply_along_axis(lambda v: O.weno5(v), -1, sr)
        return qL, qR
    return states


def test_neural_flux_enters_as_a_flux_divergence_rebuilt_independently():
    """rhs(network on) - rhs(off) = -(dF/dx + dG/dy) for F, G computed here: face images
    from WENO5 states (oracle's pinned scalar routine), frame channels, normalisation, torch's
    conv2d; y images transposed with the normal momentum first."""
    nx, ny = 10, 8
    p = W.random_periodic(nx, ny, seed=5, amp=0.2)
    U = O.prim_to_cons(p, p.W0)
    w, norm = _params(7), _norm(0.4)
    L0 = O.rhs(p, U)
    with O.neural(w, norm):
        L1 = O.rhs(p, U)
    Wp = O.cons_to_prim(p, U)
    g = p.gamma
    mean, sd, scale = norm[:4], norm[4:8], norm[8:]
    states = _faces_prim(Wp, nx, ny)

    def image(axis, n_comp, t_comp):
        qL, qR = [], []
        for c in range(4):
            a, b = states(Wp[c], axis)
            qL.append(a)
            qR.append(b)
        qL, qR = np.array(qL), np.array(qR)

        def cons(q):
            r, u, v, pr = q
            return np.stack([r, r * (u if n_comp == 1 else v), r * (v if t_comp == 2 else u),
                             pr / (g - 1) + 0.5 * r * (u * u + v * v)])
        m = 0.5 * (cons(qL) + cons(qR))
        return (m - mean[:, None, None]) / sd[:, None, None]

    Xx = image(1, 1, 2)                          # [4][ny][nx+1]
    Xy = image(0, 2, 1).transpose(0, 2, 1)       # [4][nx][ny+1]
    Fx = _torch_net(w, Xx, scale)
    Gy = _torch_net(w, Xy, scale).transpose(0, 2, 1)  # back to [4][ny+1][nx]
    Fc = np.stack([Fx[0], Fx[1], Fx[2], Fx[3]])
    Gc = np.stack([Gy[0], Gy[2], Gy[1], Gy[3]])  # normal momentum of y faces is rho v
    div = (Fc[:, :, 1:] - Fc[:, :, :-1]) / p.dx + (Gc[:, 1:, :] - Gc[:, :-1, :]) / p.dy
    diff = L1 - L0
    assert np.abs(diff + div).max() <= 1e-11 * np.abs(div).max()


def test_neural_solver_keeps_the_transpose_symmetry():
    """One shared network for both directions, y images transposed with the normal momentum
    first: the 2D step commutes with (x, y, u, v) -> (y, x, v, u)."""
    p = W.random_periodic(12, 12, seed=9, amp=0.2, mu=3e-3)
    Wt = np.stack([p.W0[0].T, p.W0[2].T, p.W0[1].T, p.W0[3].T])
    pt = p.with_(W0=Wt)
    w, norm = _params(11), _norm(0.5)
    with O.neural(w, norm):
        A = O.step(p, O.prim_to_cons(p, p.W0), [1e-3] * 2)
        Bt = O.step(pt, O.prim_to_cons(pt, Wt), [1e-3] * 2)
    back = np.stack([Bt[0].T, Bt[2].T, Bt[1].T, Bt[3].T])
    assert np.abs(back - A).max() <= 1e-14 * np.abs(A).max()


def test_weight_tangent_matches_finite_differences():
    p = W.shock_cylinder(nx=24, ny=16, Lx=3.0, Ly=2.0, centre=(1.5, 1.0), radius=0.45, x_shock=0.6, Re=100.0)
    U = O.prim_to_cons(p, W.random_state(p, seed=4, amp=0.02))
    dts = [0.2 * O.max_dt(p, U, 0.5)] * 2
    w, norm = _params(13), _norm(0.5)
    dw = np.random.default_rng(14).standard_normal(NP)
    th = O.theta_of(p)
    with O.neural(w, norm, dw=dw):
        _, dU = O.step_tangent(p, U, np.zeros_like(U), np.zeros_like(th), dts)
    # h = 1e-7: the step moves all 6388 weights at once (norm ~1e-5), larger steps cross ReLU
    # kinks of the network, where the one-sided derivative and the difference quotient differ
    h = 1e-7
    with O.neural(w + h * dw, norm):
        Up = O.step(p, U, dts)
    with O.neural(w - h * dw, norm):
        Um = O.step(p, U, dts)
    fd = (Up - Um) / (2 * h)
    assert np.abs(dU - fd).max() <= 1e-6 * np.abs(fd).max()
    assert np.abs(fd).max() > 0.0
