"""The neural flux network on the tensor cores (BF16 precision: the 16->32 and 32->4 layers as
tcgen05 implicit GEMMs, BF16 operands, FP32 accumulation) and js_nn_eval.

* js_nn_eval in FP64 equals the oracle's network; in FP32 within FP32 rounding.
* BF16: equal to a CPU emulation of the same arithmetic (torch: FP32 first layer, inputs and
  weights of layers 2 and 3 rounded to BF16, FP32 accumulation): the median difference at
  FP32 rounding, the 99th percentile within 1e-3 and every output within 1e-2 of the output
  range (a layer input on a BF16 rounding boundary may round the other way); a wrong operand
  layout gives errors of order one everywhere.  Images span several 128-pixel blocks with a
  ragged tail, a block narrower than 128 and a single row.
* The solver with the BF16 network: RHS within 3e-2 of the network's contribution of the
  oracle (FP64 network), the rest at the FP64 bar."""
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
    a1 = torch.relu(F.conv2d(x, w1, b1, padding=1))
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
