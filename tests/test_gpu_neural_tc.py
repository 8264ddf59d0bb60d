"""The neural flux network on the tensor cores (BF16 precision: the three layers of the forward
pass as tcgen05 implicit GEMMs, BF16 operands, FP32 accumulation) and js_nn_eval.

* js_nn_eval in FP64 equals the oracle's network; in FP32 within FP32 rounding.
* BF16: equal to a CPU emulation of the same arithmetic (torch: every layer's inputs and
  weights rounded to BF16, FP32 accumulation): the median difference at
  FP32 rounding, the 99th percentile within 1e-3 and every output within 1e-2 of the output
  range (a layer input on a BF16 rounding boundary may round the other way); a wrong operand
  layout gives errors of order one everywhere.  Images span several 128-pixel blocks with a
  ragged tail, a block narrower than 128 and a single row.
* The solver with the BF16 network: RHS within 3e-2 of the network's contribution of the
  oracle (FP64 network), the rest at the FP64 bar.
* js_nn_eval_vjp (the network's reverse alone): FP64 equal to torch's float64 autograd of the
  same network (itself pinned to the oracle's network on the CPU) to 1e-12, FP32 within FP32
  rounding; BF16 (data gradients of layers 3 and 2 on the tensor cores from BF16 copies of
  the output gradients, padded from 4 to 16 channels for layer 3; weight gradients of layers 3
  and 2 on the tensor cores from BF16-rounded output gradients and layer inputs, layer 1's FP32)
  equal to a CPU emulation of that arithmetic with the same bounds as the forward (a
  transposed or unflipped weight layout gives errors of order one).
* The solver's reverse in BF16 mode against its FP32 mode (which the oracle pins): the
  network's part of the state adjoint and the weight gradient within the BF16 forward's
  own deviation (its activations, tanh output and ReLU masks differ from FP32 by BF16
  rounding), the median element at the 1e-2 level."""
import numpy as np
import pytest

import oracle as O
from paper_2601_04400_gb300 import workloads as W
from jsutil import to_dev, to_host

pytestmark = pytest.mark.gpu

NP = 6388


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04400_gb300 import binding as B
    B.lib()
    return torch, B


def _params(seed, amp=0.2):
    return np.random.default_rng(seed).standard_normal(NP) * amp


NORM = np.concatenate([[1.0, 0.1, 0.05, 2.5], [0.3, 0.4, 0.4, 0.8], [0.5, 0.4, 0.3, 0.6]])


def _solver(B, nx=64, ny=48):
    return B.Solver.from_problem(W.random_periodic(nx, ny, seed=0))


def _emulate_bf16(torch, w, X, scale):
    import torch.nn.functional as F
    t = torch.tensor(w, dtype=torch.float32)
    w1, b1 = t[:576].view(16, 4, 3, 3), t[576:592]
    w2, b2 = t[592:5200].view(32, 16, 3, 3), t[5200:5232]
    w3, b3 = t[5232:6384].view(4, 32, 3, 3), t[6384:]
    bf = lambda a: a.to(torch.bfloat16).to(torch.float32)
    x = torch.tensor(X, dtype=torch.float32)[None]
    a1 = torch.relu(F.conv2d(bf(x), bf(w1), b1, padding=1))
    a2 = torch.relu(F.conv2d(bf(a1), bf(w2), b2, padding=1))
    z3 = F.conv2d(bf(a2), bf(w3), b3, padding=1)
    return (torch.tensor(scale, dtype=torch.float32)[:, None, None] * torch.tanh(z3[0])).double().numpy()


SHAPES = [(17, 300), (9, 37), (1, 201)]


@pytest.mark.parametrize("shape", SHAPES)
def test_nn_eval_fp64_and_fp32_match_oracle(env, shape):
    torch, B = env
    w = _params(1)
    X = np.random.default_rng(2).standard_normal((4,) + shape)
    with O.neural(w, NORM):
        ref = O.nn_eval(X)
    s = _solver(B)
    wd = torch.tensor(w, device="cuda")
    for prec, tol in (("fp64", 1e-12), ("fp32", 2e-5)):
        s.set_neural(wd, NORM, precision=prec)
        Y = to_host(s.nn_eval(to_dev(X)))
        assert np.abs(Y - ref).max() <= tol * np.abs(ref).max(), prec
    assert s.status() == 0


@pytest.mark.parametrize("shape", SHAPES)
def test_bf16_tensor_core_layers_match_emulation(env, shape):
    torch, B = env
    w = _params(3)
    X = np.random.default_rng(4).standard_normal((4,) + shape)
    s = _solver(B)
    s.set_neural(torch.tensor(w, device="cuda"), NORM, precision="bf16")
    Y = to_host(s.nn_eval(to_dev(X)))
    assert s.status() == 0
    emu = _emulate_bf16(torch, w, X, NORM[8:])
    span = np.abs(emu).max()
    d = np.abs(Y - emu)
    # almost every output equals the emulation to FP32 accumulation rounding; a layer input that
    # sits on a BF16 rounding boundary may round the other way (one BF16 step, 2^-8 relative)
    assert np.median(d) <= 1e-5 * span and np.quantile(d, 0.99) <= 1e-3 * span
    assert d.max() <= 1e-2 * span
    with O.neural(w, NORM):
        ref = O.nn_eval(X)
    # BF16 against the exact network: of the order of the BF16 rounding of 144- and 288-term
    # dot products (the emulation itself is up to 5% of the range off for these weights)
    e = np.abs(Y - ref)
    assert np.quantile(e, 0.99) <= 3e-2 * np.abs(ref).max() and e.max() <= 1e-1 * np.abs(ref).max()


def test_bf16_solver_rhs_within_bound(env):
    torch, B = env
    p = W.shock_cylinder(nx=70, ny=45, Lx=3.5, Ly=2.25, centre=(1.6, 1.1), radius=0.45, x_shock=0.8, viscous=False)
    U = O.prim_to_cons(p, W.random_state(p, seed=2, amp=0.02))
    w = _params(5, amp=0.12)
    s = B.Solver.from_problem(p)
    s.set_neural(torch.tensor(w, device="cuda"), NORM, precision="bf16")
    with O.neural(w, NORM):
        L_ref = O.rhs(p, U)
    part = np.abs(L_ref - O.rhs(p, U)).max()
    err = np.abs(to_host(s.rhs(to_dev(U))) - L_ref).max()
    assert s.status() == 0
    assert part > 0 and err <= 3e-2 * part + 1e-10 * np.abs(L_ref).max(), (err, part)


@pytest.mark.parametrize("viscous", [False, True])
def test_bf16_reverse_matches_fp32_reverse(env, viscous):
    torch, B = env
    p = W.shock_cylinder(nx=70, ny=45, Lx=3.5, Ly=2.25, centre=(1.6, 1.1), radius=0.45, x_shock=0.8,
                         viscous=viscous)
    U = to_dev(O.prim_to_cons(p, W.random_state(p, seed=2, amp=0.02)))
    lam = to_dev(np.random.default_rng(6).standard_normal((4, p.ny, p.nx)))
    w = torch.tensor(_params(5, amp=0.12), device="cuda")
    s = B.Solver.from_problem(p)
    dt = 0.3 * s.max_dt(U, 0.5)
    off, _ = s.rhs_vjp(U, lam)
    off_step, _ = s.step_vjp(U, dt, lam)
    out = {}
    for prec in ("fp32", "bf16"):
        wb = torch.zeros(NP, dtype=torch.float64, device="cuda")
        s.set_neural(w, NORM, w_bar=wb, precision=prec)
        Ub, pb = s.rhs_vjp(U, lam)
        wb2 = torch.zeros_like(wb)
        s.set_neural(w, NORM, w_bar=wb2, precision=prec)
        ls, _ = s.step_vjp(U, dt, lam)
        out[prec] = (to_host(Ub), to_host(wb), to_host(ls), to_host(wb2))
        assert s.status() == 0
    net = np.abs(out["fp32"][0] - to_host(off)).max()
    net_step = np.abs(out["fp32"][2] - to_host(off_step)).max()
    assert net > 0 and net_step > 0
    for k, ref_scale in ((0, net), (1, None), (2, net_step), (3, None)):
        a, b = out["bf16"][k], out["fp32"][k]
        scale = ref_scale if ref_scale is not None else np.abs(b).max()
        d = np.abs(a - b)
        assert d.max() <= 0.25 * scale, (k, d.max() / scale)
        assert np.median(d) <= 1e-2 * scale, (k, np.median(d) / scale)


def _torch_net(torch, w, dtype):
    t = torch.tensor(w, dtype=dtype)
    return (t[:576].view(16, 4, 3, 3), t[576:592], t[592:5200].view(32, 16, 3, 3), t[5200:5232],
            t[5232:6384].view(4, 32, 3, 3), t[6384:])


def _grads_flat(dw1, db1, dw2, db2, dw3, db3):
    return np.concatenate([x.reshape(-1).double().numpy() for x in (dw1, db1, dw2, db2, dw3, db3)])


def _autograd_vjp(torch, w, X, GY, scale):
    import torch.nn.functional as F
    ps = [p.clone().requires_grad_(True) for p in _torch_net(torch, w, torch.float64)]
    x = torch.tensor(X, dtype=torch.float64, requires_grad=True)
    a1 = torch.relu(F.conv2d(x[None], ps[0], ps[1], padding=1))
    a2 = torch.relu(F.conv2d(a1, ps[2], ps[3], padding=1))
    y = torch.tensor(scale, dtype=torch.float64)[:, None, None] * torch.tanh(F.conv2d(a2, ps[4], ps[5], padding=1)[0])
    g = torch.autograd.grad(y, [x] + ps, torch.tensor(GY, dtype=torch.float64))
    return g[0].numpy(), _grads_flat(*g[1:])


def _emulate_bf16_vjp(torch, w, X, GY, scale):
    """The BF16 mode's reverse, rounding where the kernels round (FP32 elsewhere)."""
    import torch.nn.functional as F
    from torch.nn.grad import conv2d_input, conv2d_weight
    w1, b1, w2, b2, w3, b3 = _torch_net(torch, w, torch.float32)
    bf = lambda a: a.to(torch.bfloat16).to(torch.float32)
    x = torch.tensor(X, dtype=torch.float32)[None]
    a1 = torch.relu(F.conv2d(bf(x), bf(w1), b1, padding=1))
    a2 = torch.relu(F.conv2d(bf(a1), bf(w2), b2, padding=1))
    t3 = torch.tanh(F.conv2d(bf(a2), bf(w3), b3, padding=1))
    g4 = (torch.tensor(GY, dtype=torch.float64)[None] * torch.tensor(scale, dtype=torch.float64)[:, None, None]
          * (1.0 - t3.double() ** 2)).float()
    g32 = conv2d_input(a2.shape, bf(w3), bf(g4), padding=1) * (a2 > 0)
    g16 = conv2d_input(a1.shape, bf(w2), bf(g32), padding=1) * (a1 > 0)
    gx = conv2d_input(x.shape, w1, g16, padding=1)
    # weight gradients of layers 3 and 2 on the tensor cores (output gradients and layer inputs
    # rounded to BF16), layer 1's in FP32
    dw3 = conv2d_weight(bf(a2), w3.shape, bf(g4), padding=1)
    dw2 = conv2d_weight(bf(a1), w2.shape, bf(g32), padding=1)
    dw1 = conv2d_weight(x, w1.shape, g16, padding=1)
    return gx[0].double().numpy(), _grads_flat(dw1, g16.sum((0, 2, 3)), dw2, bf(g32).sum((0, 2, 3)), dw3,
                                               bf(g4).sum((0, 2, 3)))


@pytest.mark.parametrize("shape", SHAPES)
def test_nn_eval_vjp_fp64_fp32_and_bf16(env, shape):
    torch, B = env
    w = _params(7)
    rng = np.random.default_rng(8)
    X = rng.standard_normal((4,) + shape)
    GY = rng.standard_normal((4,) + shape)
    gx_ref, gw_ref = _autograd_vjp(torch, w, X, GY, NORM[8:])
    s = _solver(B)
    wd = torch.tensor(w, device="cuda")
    for prec, tol in (("fp64", 1e-12), ("fp32", 2e-4)):
        wb = torch.zeros(NP, dtype=torch.float64, device="cuda")
        s.set_neural(wd, NORM, w_bar=wb, precision=prec)
        gx = to_host(s.nn_eval_vjp(to_dev(X), to_dev(GY)))
        assert np.abs(gx - gx_ref).max() <= tol * np.abs(gx_ref).max(), prec
        assert np.abs(to_host(wb) - gw_ref).max() <= tol * np.abs(gw_ref).max(), prec
    wb = torch.zeros(NP, dtype=torch.float64, device="cuda")
    s.set_neural(wd, NORM, w_bar=wb, precision="bf16")
    gx = to_host(s.nn_eval_vjp(to_dev(X), to_dev(GY)))
    gb = to_host(wb)
    assert s.status() == 0
    ex, ew = _emulate_bf16_vjp(torch, w, X, GY, NORM[8:])
    span = np.abs(ex).max()
    d = np.abs(gx - ex)
    assert np.median(d) <= 1e-5 * span and np.quantile(d, 0.99) <= 1e-3 * span, (np.median(d) / span,
                                                                                   np.quantile(d, 0.99) / span)
    assert d.max() <= 1e-2 * span, d.max() / span
    dw = np.abs(gb - ew)
    assert dw.max() <= 1e-3 * np.abs(ew).max(), dw.max() / np.abs(ew).max()
    # and against the exact reverse: of the order of BF16 rounding (every layer's inputs and weights
    # rounded to BF16 in the forward, whose ReLU masks the reverse applies: a few percent)
    assert np.quantile(np.abs(gx - gx_ref), 0.99) <= 1e-1 * np.abs(gx_ref).max()


# The fused network kernel (one launch for the three layers of a forward-only BF16 stage) runs the
# arithmetic of the layer-by-layer launches in the same order: equal bit for bit.  Images with
# several 124-pixel strips and a ragged one, bands with a ragged last band, a single row, an image
# narrower than one strip, and the 1024 x 1024 solver at full size.
FUSED_SHAPES = [(17, 300), (9, 37), (1, 201), (130, 250), (300, 129), (64, 125)]


@pytest.mark.parametrize("shape", FUSED_SHAPES)
def test_fused_network_equals_layerwise_launches(env, shape):
    torch, B = env
    w = _params(11)
    X = np.random.default_rng(12).standard_normal((4,) + shape)
    s = B.Solver.from_problem(W.random_periodic(256, 200, seed=0))
    wd = torch.tensor(w, device="cuda")
    out = {}
    for prec in ("bf16", "bf16-layerwise"):
        s.set_neural(wd, NORM, precision=prec)
        out[prec] = to_host(s.nn_eval(to_dev(X)))
    assert s.status() == 0
    assert np.array_equal(out["bf16"], out["bf16-layerwise"])
    assert np.abs(out["bf16"]).max() > 0


@pytest.mark.parametrize("n", [96, 1024, "sod"])
def test_fused_network_solver_steps_equal_layerwise(env, n):
    torch, B = env
    from paper_2601_04400_gb300 import neural as NN
    p = W.sod(200) if n == "sod" else W.riemann2d(n)  # sod: one image, one row high
    U0 = to_dev(O.prim_to_cons(p, p.W0))
    # the benchmark's network: He-uniform weights, outputs scaled to a tenth of the states' spread
    w = NN.init_weights(0, zero_last=False) * 0.5
    norm = NN.frame_norm(U0, scale=0.1)
    res = {}
    for prec in ("bf16", "bf16-layerwise"):
        s = B.Solver.from_problem(p)
        dt = s.max_dt(U0, 0.3)
        s.set_neural(w, norm, precision=prec)
        U = U0.clone()
        L = s.rhs(U)
        s.step(U, dt, 3)
        res[prec] = (to_host(L), to_host(U), s.status())
        s.close()
    assert res["bf16"][2] == 0 and res["bf16-layerwise"][2] == 0, (res["bf16"][2], res["bf16-layerwise"][2])
    for a, b in zip(res["bf16"][:2], res["bf16-layerwise"][:2]):
        assert np.array_equal(a, b)


# Forward stages write the network's face images from the stage kernel's own WENO5 face states;
# stages that store their WENO5 internals (for a reverse pass) form them in a separate kernel from
# those internals.  The two routes share the face-image arithmetic: equal stage outputs bit for
# bit, for Euler and Navier-Stokes stage kernels, on a grid that is not a multiple of the tile.
@pytest.mark.parametrize("prec", ["bf16", "fp32"])
@pytest.mark.parametrize("case", ["riemann", "cylinder"])
def test_stage_kernel_images_equal_image_kernel(env, prec, case):
    torch, B = env
    from paper_2601_04400_gb300 import neural as NN
    if case == "riemann":
        p = W.riemann2d(70, ny=45)
    else:
        p = W.shock_cylinder(nx=70, ny=45, Lx=3.5, Ly=2.25, centre=(1.6, 1.1), radius=0.45, x_shock=0.8,
                             viscous=True)
    U0 = to_dev(O.prim_to_cons(p, W.random_state(p, seed=3, amp=0.02)))
    s = B.Solver.from_problem(p)
    dt = s.max_dt(U0, 0.3)
    s.set_neural(NN.init_weights(0, zero_last=False) * 0.5, NN.frame_norm(U0, scale=0.1), precision=prec)
    out = {}
    for internals in (False, True):
        U1, U2 = torch.empty_like(U0), torch.empty_like(U0)
        s.step_stage(U0, U0, U1, dt, 0, internals=internals)
        s.step_stage(U0, U1, U2, dt, 1, internals=internals)
        out[internals] = (to_host(U1), to_host(U2))
    assert s.status() == 0
    for a, b in zip(out[False], out[True]):
        assert np.array_equal(a, b)
