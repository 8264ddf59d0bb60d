"""The hand-written reverse mode (js_rhs_vjp, js_step_vjp) against the oracle's discrete
derivative (forward-mode dual numbers through the same FP64 formulation): the full
transposed Jacobian on small grids, column by column, for every boundary kind, the viscous
terms, artificial viscosity and the immersed cylinder; parameter gradients for gamma, mu,
Pr, nu and the inflow states; dot-product tests on larger grids."""
import numpy as np
import pytest

import oracle as O
from paper_2601_04400_gb300 import workloads as W
from jsutil import to_dev, to_host

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04400_gb300 import binding
    binding.lib()
    return binding


def _small_cases():
    out = []
    p = W.random_periodic(12, 10, seed=1)
    out.append(("euler_periodic_12x10", p, p.W0))
    p = W.random_periodic(12, 10, seed=2, mu=5e-3, nu=1e-3)
    out.append(("ns_av_periodic_12x10", p, p.W0))
    p = W.random_periodic(11, 9, seed=3, mu=2e-3).with_(bc=(3, 1, 0, 3), inflow=np.array(
        [[1.1, 0.3, 0.1, 0.9], [1.0, 0.0, 0.0, 1.0], [1.0, 0.0, 0.0, 1.0], [1.2, -0.1, -0.2, 0.8]]))
    out.append(("mixed_inflow_reflective_11x9", p, p.W0))
    p = W.sod(16)
    out.append(("sod16", p, W.random_state(p, seed=4, amp=0.02)))
    p = W.shock_cylinder(nx=24, ny=16, mach=2.0, Re=100.0, Lx=3.0, Ly=2.0, centre=(1.5, 1.0), radius=0.45,
                         x_shock=0.6)
    out.append(("cylinder_ns_24x16", p, W.random_state(p, seed=5, amp=0.02)))
    p = W.shock_cylinder(nx=24, ny=16, mach=2.0, viscous=False, Lx=3.0, Ly=2.0, centre=(1.5, 1.0), radius=0.45,
                         x_shock=0.6).with_(wall=1)
    out.append(("cylinder_noslip_euler_24x16", p, W.random_state(p, seed=6, amp=0.02)))
    # contact discontinuities at rest (u = v = 0, uniform p, random density): s* = 0 exactly
    # at every face, where the flux is the average of both HLLC branches and its derivative
    # the average of the branches' derivatives
    p = W.random_periodic(12, 10, seed=7)
    Wc = p.W0.copy()
    Wc[1:3] = 0.0
    Wc[3] = 1.0
    out.append(("contact_at_rest_periodic_12x10", p, Wc))
    # the unperturbed shock-cylinder initial condition: quiescent gas ahead of the shock
    p = W.shock_cylinder(nx=24, ny=16, mach=2.0, Re=100.0, Lx=3.0, Ly=2.0, centre=(1.5, 1.0), radius=0.45,
                         x_shock=0.6)
    out.append(("cylinder_ns_initial_24x16", p, p.W0))
    return out


SMALL = _small_cases()


def _oracle_vjp(prob, U, lam, tangent_fn):
    """(J^T lam, dL/dtheta . lam) column by column from the oracle's forward mode."""
    n = U.size
    Ub = np.zeros(n)
    e = np.zeros(n)
    dth0 = np.zeros(20)
    for k in range(n):
        e[k] = 1.0
        dL = tangent_fn(e.reshape(U.shape), dth0)
        Ub[k] = np.dot(lam.reshape(-1), dL.reshape(-1))
        e[k] = 0.0
    pb = np.zeros(20)
    zero = np.zeros_like(U)
    for k in range(20):
        d = np.zeros(20)
        d[k] = 1.0
        pb[k] = np.dot(lam.reshape(-1), tangent_fn(zero, d).reshape(-1))
    return Ub.reshape(U.shape), pb


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _pbar_ok(got, ref, m, lam, prob):
    """Parameter gradients within TOL of the oracle's, relative to its largest entry; a gradient
    that vanishes exactly (the contact at rest: its fluxes do not depend on gamma) must vanish
    to round-off of the summed face terms, |lambda|_1 / h times 1e-12."""
    scale = np.abs(ref[m]).max()
    if scale == 0.0:
        return np.abs(got[m]).max() <= 1e-12 * np.abs(lam).sum() / min(prob.dx, prob.dy)
    return np.abs(got[m] - ref[m]).max() <= TOL * scale


def _pbar_mask(prob):
    """Parameters whose gradient the library computes for this problem: gamma always; mu and
    Pr for viscous problems (mu > 0); nu when the artificial viscosity is on (nu > 0); the
    inflow state of inflow sides."""
    m = np.zeros(20, dtype=bool)
    m[0] = True
    if prob.mu > 0:
        m[1] = m[2] = True
    if prob.nu > 0:
        m[3] = True
    for s in range(4):
        if prob.bc[s] == 3 and not (prob.ny == 1 and s >= 2):
            m[4 + 4 * s:8 + 4 * s] = True
    return m


@pytest.mark.parametrize("name,prob,Wp", SMALL, ids=[c[0] for c in SMALL])
def test_rhs_vjp_equals_oracle_transposed_jacobian(B, name, prob, Wp):
    import torch
    U = O.prim_to_cons(prob, Wp)
    lam = W.uniform_normal(U.shape, seed=11)
    ref_U, ref_p = _oracle_vjp(prob, U, lam, lambda dU, dth: O.rhs_tangent(prob, U, dU, dth)[1])
    s = B.Solver.from_problem(prob)
    Ub, pb = s.rhs_vjp(to_dev(U), to_dev(lam))
    assert s.status() == 0
    assert _rel(to_host(Ub), ref_U) < TOL
    assert _pbar_ok(to_host(pb), ref_p, _pbar_mask(prob), lam, prob)


@pytest.mark.parametrize("name,prob,Wp", SMALL, ids=[c[0] for c in SMALL])
def test_step_vjp_equals_oracle_transposed_jacobian(B, name, prob, Wp):
    U = O.prim_to_cons(prob, Wp)
    dt = 0.4 * O.max_dt(prob, U, 0.5)
    lam = W.uniform_normal(U.shape, seed=12)
    ref_U, ref_p = _oracle_vjp(prob, U, lam, lambda dU, dth: O.step_tangent(prob, U, dU, dth, [dt])[1])
    s = B.Solver.from_problem(prob)
    Ub, pb = s.step_vjp(to_dev(U), dt, to_dev(lam))
    assert s.status() == 0
    assert _rel(to_host(Ub), ref_U) < TOL
    assert _pbar_ok(to_host(pb), ref_p, _pbar_mask(prob), lam, prob)


@pytest.mark.parametrize("which", ["cylinder_ns_96x64", "riemann_ragged_70x45", "sod200"])
def test_step_vjp_dot_product(B, which):
    """<lam, J v> from the oracle's tangent equals <J^T lam, v> from the GPU on larger grids."""
    if which == "cylinder_ns_96x64":
        prob = W.shock_cylinder(nx=96, ny=64, Lx=6.0, Ly=4.0, Re=300.0)
    elif which == "riemann_ragged_70x45":
        prob = W.riemann2d(70, ny=45)
    else:
        prob = W.sod(200)
    U = O.prim_to_cons(prob, W.random_state(prob, seed=7, amp=0.02))
    dt = 0.4 * O.max_dt(prob, U, 0.5)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(U.shape) * np.abs(U).max(axis=(1, 2), keepdims=True) * 1e-3
    dth = np.zeros(20)
    dth[0] = 0.1
    if prob.mu > 0:
        dth[1] = 1e-3
    lam = rng.standard_normal(U.shape)
    _, Jv = O.step_tangent(prob, U, v, dth, [dt])
    s = B.Solver.from_problem(prob)
    Ub, pb = s.step_vjp(to_dev(U), dt, to_dev(lam))
    lhs = np.dot(lam.reshape(-1), Jv.reshape(-1))
    rhs = np.dot(to_host(Ub).reshape(-1), v.reshape(-1)) + np.dot(to_host(pb), dth)
    scale = np.abs(lam).sum() * np.abs(Jv).max()
    assert abs(lhs - rhs) <= 1e-12 * scale


def test_taped_step_and_vjp_equal_the_recomputing_ones(B):
    prob = W.shock_cylinder(nx=96, ny=64, Lx=6.0, Ly=4.0, Re=300.0)
    U = O.prim_to_cons(prob, W.random_state(prob, seed=9, amp=0.02))
    dt = 0.4 * O.max_dt(prob, U, 0.5)
    lam = W.uniform_normal(U.shape, seed=13)
    s = B.Solver.from_problem(prob)
    s.tape_reserve(3)
    Ut, Ur = to_dev(U), to_dev(U)
    s.step_taped(Ut, dt, 2)
    s.step(Ur, dt, 1)
    assert np.array_equal(to_host(Ut), to_host(Ur))
    lt, pt = s.step_vjp_taped(2, dt, to_dev(lam))
    lr, pr = s.step_vjp(to_dev(U), dt, to_dev(lam))
    assert s.status() == 0
    assert np.abs(to_host(lt) - to_host(lr)).max() <= 1e-12 * np.abs(to_host(lr)).max()
    assert np.abs(to_host(pt) - to_host(pr)).max() <= 1e-12 * np.abs(to_host(pr)).max()


@pytest.mark.parametrize("shape", [(48, 32), (32, 48), (37, 21)])
@pytest.mark.parametrize("viscous", [False, True])
def test_reverse_with_forward_stored_weno_internals(B, shape, viscous):
    """The WENO5 internals stored by the forward stage (js_step_vjp's stages 1-2, a tape with
    JS_TAPE_WENO) give the same reverse step as recomputing them in pass 1 (a tape without
    internals).  48 and 32 cells put a segment end on the last cell of a line; 48 also has
    two writers of that cell; 37 x 21 is ragged."""
    nx, ny = shape
    if viscous:
        prob = W.shock_cylinder(nx=nx, ny=ny, Lx=nx / 16.0, Ly=ny / 16.0, centre=(nx / 32.0, ny / 32.0),
                                radius=min(nx, ny) / 64.0, x_shock=nx / 64.0, Re=200.0)
    else:
        prob = W.random_periodic(nx, ny, seed=21)
    U = O.prim_to_cons(prob, W.random_state(prob, seed=5, amp=0.02))
    dt = 0.4 * O.max_dt(prob, U, 0.5)
    lam = W.uniform_normal(U.shape, seed=17)
    s = B.Solver.from_problem(prob)
    s.tape_reserve(2, weno=False)
    Ua = to_dev(U)
    s.step_taped(Ua, dt, 0)
    l0, p0 = s.step_vjp_taped(0, dt, to_dev(lam))     # pass 1 recomputes every stage
    s.tape_reserve(2, weno=True)
    Ub = to_dev(U)
    s.step_taped(Ub, dt, 1)
    assert np.array_equal(to_host(Ua), to_host(Ub))
    l1, p1 = s.step_vjp_taped(1, dt, to_dev(lam))     # all three stages from the tape
    l2, p2 = s.step_vjp(to_dev(U), dt, to_dev(lam))   # stages 1-2 stored, stage 3 recomputed
    assert s.status() == 0
    ref, pref = to_host(l0), to_host(p0)
    for l, p in ((l1, p1), (l2, p2)):
        # summation order of the atomics is the only difference
        assert np.abs(to_host(l) - ref).max() <= 1e-12 * np.abs(ref).max()
        assert np.abs(to_host(p) - pref).max() <= 1e-12 * max(np.abs(pref).max(), 1e-300)


# ---------------------------------------------------------------------------------------
# the reverse pass is deterministic: no floating-point atomics, every sum in a fixed order
# ---------------------------------------------------------------------------------------
def _det_cases():
    out = []
    p = W.adjoint_case(512)
    out.append(("adjoint_case_512", p, W.random_state(p, seed=11, amp=0.02), None))
    p = W.random_periodic(96, 64, seed=4, mu=3e-3, nu=2e-4)
    out.append(("periodic_ns_av_96x64", p, p.W0, None))
    p = W.mach5_cylinder(nx=218, ny=97)
    out.append(("mach5_fallback_218x97", p, p.W0, None))  # positivity fallback faces
    p = W.random_periodic(40, 33, seed=5).with_(bc=(3, 1, 0, 3), mu=1e-3, inflow=np.array(
        [[1.1, 0.3, 0.1, 0.9], [1.0, 0.0, 0.0, 1.0], [1.0, 0.0, 0.0, 1.0], [1.2, -0.1, -0.2, 0.8]]))
    out.append(("mixed_inflow_40x33", p, p.W0, None))
    p = W.sod(200)
    out.append(("sod200", p, p.W0, None))
    p = W.shock_cylinder(nx=128, ny=64)
    out.append(("cylinder_neural_128x64", p, W.random_state(p, seed=7, amp=0.02), "fp64"))
    return out


DET = _det_cases()


@pytest.mark.parametrize("name,prob,Wp,nn", DET, ids=[c[0] for c in DET])
def test_reverse_step_is_bitwise_reproducible(B, name, prob, Wp, nn):
    """js_step_vjp twice (and the taped reverse twice) on the same inputs: lambda_n and p_bar
    equal bit for bit."""
    import torch
    s = B.Solver.from_problem(prob)
    U = to_dev(O.prim_to_cons(prob, Wp))
    if nn:
        from paper_2601_04400_gb300 import neural as NN
        w = NN.init_weights(0, zero_last=False) * 0.5
        wb = torch.zeros_like(w)
        s.set_neural(w, NN.frame_norm(U, scale=0.1), w_bar=wb, precision=nn)
    dt = 0.5 * s.max_dt(U, prob.cfl)
    lam = to_dev(W.uniform_normal(U.shape, seed=3))
    outs = []
    for _ in range(2):
        pb = torch.zeros(20, dtype=torch.float64, device="cuda")
        ln, _ = s.step_vjp(U, dt, lam, p_bar=pb)
        outs.append((to_host(ln), to_host(pb)))
    assert s.status() == 0
    assert outs[0][0].tobytes() == outs[1][0].tobytes()
    assert outs[0][1].tobytes() == outs[1][1].tobytes()
    assert np.abs(outs[0][1]).max() > 0
    if not nn:
        s.tape_reserve(1, weno=prob.ny > 1)
        tap = []
        for _ in range(2):
            Ut = U.clone()
            s.step_taped(Ut, dt, 0)
            pb = torch.zeros(20, dtype=torch.float64, device="cuda")
            ln, _ = s.step_vjp_taped(0, dt, lam, p_bar=pb)
            tap.append((to_host(ln), to_host(pb)))
        assert tap[0][0].tobytes() == tap[1][0].tobytes() and tap[0][1].tobytes() == tap[1][1].tobytes()
    s.close()
