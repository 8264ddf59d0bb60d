"""Pins of the FP64 CPU oracle against facts that do not come from the oracle itself:
values the paper prints, textbook closed forms, conservation and symmetry invariants,
polynomial exactness, brute-force integrals and finite differences.  CPU only.
"""
import numpy as np
import pytest

import oracle as O
from paper_2601_04400_gb300 import workloads as W
from conftest import golden


# ---------------------------------------------------------------------------------------
# exact Riemann solver and the Sod case (Sec. 3)
# ---------------------------------------------------------------------------------------
def _sod_inputs():
    g = golden("paper_sod_states.txt")[0]
    return (g[0], g[1], g[2]), (g[3], g[4], g[5]), g[6], g[7]


def test_exact_riemann_matches_textbook_star_state():
    left, right, gamma, t = _sod_inputs()
    _, _, _, star = O.exact_riemann(left, right, gamma, np.array([0.5]), 0.5, t)
    ref = golden("toro_sod_star.txt")[0]
    got = np.array([star["p"], star["u"], star["rhoL"], star["rhoR"]])
    assert np.allclose(got, ref, rtol=0, atol=6e-6)


def test_exact_riemann_satisfies_jump_conditions():
    """Independent of any table: Rankine-Hugoniot across the right shock, isentrope and
    Riemann invariant across the left rarefaction, equal p and u across the contact."""
    (rl, ul, pl), (rr, ur, pr), g, t = _sod_inputs()
    _, _, _, s = O.exact_riemann((rl, ul, pl), (rr, ur, pr), g, np.array([0.5]), 0.5, t)
    p, u, rsl, rsr = s["p"], s["u"], s["rhoL"], s["rhoR"]
    # right-moving shock with speed S: mass, momentum and energy fluxes continuous
    S = (rsr * u - rr * ur) / (rsr - rr)
    E = lambda r, v, pp: pp / (g - 1) + 0.5 * r * v * v
    m1 = rr * (ur - S)
    m2 = rsr * (u - S)
    assert abs(m1 - m2) < 1e-12
    assert abs((rr * ur * (ur - S) + pr) - (rsr * u * (u - S) + p)) < 1e-12
    assert abs(((E(rr, ur, pr) + pr) * ur - S * E(rr, ur, pr)) - ((E(rsr, u, p) + p) * u - S * E(rsr, u, p))) < 1e-12
    # left rarefaction: isentropic and u + 2a/(g-1) constant
    assert abs(p / rsl ** g - pl / rl ** g) < 1e-12
    a = lambda r, pp: np.sqrt(g * pp / r)
    assert abs((ul + 2 * a(rl, pl) / (g - 1)) - (u + 2 * a(rsl, p) / (g - 1))) < 1e-12


def test_sod_converges_to_exact_solution():
    left, right, gamma, t = _sod_inputs()
    errs = []
    for n in (100, 200, 400):
        p = W.sod(n, t_end=t)
        U, dts = O.run_to(p, O.prim_to_cons(p, p.W0), 0.5, t)
        assert abs(dts.sum() - t) < 1e-14
        x = (np.arange(n) + 0.5) / n
        r, u, pp, _ = O.exact_riemann(left, right, gamma, x, 0.5, t)
        Wf = O.cons_to_prim(p, U)
        errs.append(np.mean(np.abs(Wf[0, 0] - r)))
        if n == 200:
            # calibrated bound: WENO5-HLLC-RK3 at N = 200 (measured 2.44e-3)
            assert errs[-1] < 3.0e-3
            assert np.mean(np.abs(Wf[3, 0] - pp)) < 2.5e-3
            assert np.mean(np.abs(Wf[1, 0] - u)) < 6.0e-3
    assert errs[0] > errs[1] > errs[2]


# ---------------------------------------------------------------------------------------
# WENO5
# ---------------------------------------------------------------------------------------
def _cell_averages_of_poly(coef, centres, h):
    """Exact cell averages of sum coef[k] x^k over [c - h/2, c + h/2]."""
    P = np.polynomial.polynomial
    anti = P.polyint(coef)
    return (P.polyval(centres + h / 2, anti) - P.polyval(centres - h / 2, anti)) / h


def test_weno_linear_weights_reproduce_quartics():
    rng = np.random.default_rng(1)
    P = np.polynomial.polynomial
    for deg in range(5):
        for _ in range(20):
            coef = rng.standard_normal(deg + 1)
            h = rng.uniform(0.05, 0.5)
            c = np.arange(-2, 3) * h
            avg = _cell_averages_of_poly(coef, c, h)
            exact = P.polyval(h / 2, coef)  # right edge of the centre cell
            got = O.weno5(avg, linear=True)
            assert abs(got - exact) <= 1e-12 * max(1.0, np.abs(avg).max())
            # mirrored stencil gives the left edge
            got_l = O.weno5(avg[::-1], linear=True)
            assert abs(got_l - P.polyval(-h / 2, coef)) <= 1e-12 * max(1.0, np.abs(avg).max())


def test_weno_smoothness_indicators_are_the_jiang_shu_integrals():
    """beta_k = sum_l h^(2l-1) int_cell (d^l P_k / dx^l)^2 dx with P_k the quadratic whose cell
    averages match stencil k; brute-force construction with numpy, h = 1."""
    rng = np.random.default_rng(2)
    P = np.polynomial.polynomial
    for _ in range(50):
        q = rng.standard_normal(5) * rng.uniform(0.1, 10)
        beta = O.weno5_beta(q)
        for k in range(3):
            cells = np.array([k - 2, k - 1, k], dtype=float)  # centres relative to the target cell
            A = np.array([[(((c + 0.5) ** (m + 1) - (c - 0.5) ** (m + 1)) / (m + 1)) for m in range(3)]
                          for c in cells])
            coef = np.linalg.solve(A, q[k:k + 3])
            d1, d2 = P.polyder(coef, 1), P.polyder(coef, 2)
            i1 = P.polyint(P.polymul(d1, d1))
            i2 = P.polyint(P.polymul(d2, d2))
            ref = (P.polyval(0.5, i1) - P.polyval(-0.5, i1)) + (P.polyval(0.5, i2) - P.polyval(-0.5, i2))
            assert abs(beta[k] - ref) <= 1e-11 * max(1.0, abs(ref))


def test_weno_is_non_oscillatory_at_a_step():
    for lo, hi in ((0.0, 1.0), (1.0, 0.125), (-3.0, 2.0)):
        for cut in range(1, 5):
            q = np.array([lo] * cut + [hi] * (5 - cut))
            v = O.weno5(q)
            assert min(lo, hi) - 1e-9 * abs(hi - lo) <= v <= max(lo, hi) + 1e-9 * abs(hi - lo)


def test_rhs_is_fifth_order_on_smooth_wave():
    errs = []
    for n in (32, 64, 128, 256):
        p = W.smooth_wave(n)
        L = O.rhs(p, O.prim_to_cons(p, p.W0))
        dx = 1.0 / n
        x = (np.arange(n) + 0.5) * dx
        amp = p.meta["amp"]
        exact = -amp * (np.sin(2 * np.pi * (x + 0.5 * dx)) - np.sin(2 * np.pi * (x - 0.5 * dx))) / dx
        errs.append(np.mean(np.abs(L[0, 0] - exact)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 4.8, orders


def test_full_step_is_fifth_order_with_dt_scaled():
    errs = []
    T = 0.1
    for n in (20, 40, 80):
        p = W.smooth_wave(n)
        dx = 1.0 / n
        dt = 0.25 * dx * (dx / 0.05) ** (2.0 / 3.0)
        nst = int(np.ceil(T / dt))
        U = O.step(p, O.prim_to_cons(p, p.W0), np.full(nst, T / nst))
        x = (np.arange(n) + 0.5) * dx
        amp = p.meta["amp"]
        exact = 1 + amp * (np.cos(2 * np.pi * (x - T - 0.5 * dx)) - np.cos(2 * np.pi * (x - T + 0.5 * dx))) / (2 * np.pi * dx)
        errs.append(np.mean(np.abs(U[0, 0] - exact)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 4.8, orders


# ---------------------------------------------------------------------------------------
# HLLC (Sec. 2)
# ---------------------------------------------------------------------------------------
def _rand_state(rng):
    return np.array([rng.uniform(0.1, 5), rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(0.05, 10)])


def _phys_flux(q, g):
    r, u, v, p = q
    E = p / (g - 1) + 0.5 * r * (u * u + v * v)
    return np.array([r * u, r * u * u + p, r * u * v, u * (E + p)]), np.array([r, r * u, r * v, E])


def test_hllc_star_states_satisfy_integral_consistency():
    """(s*-sL) U*L + (sR-s*) U*R = sR UR - sL UL - (FR - FL)."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        qL, qR, g = _rand_state(rng), _rand_state(rng), rng.uniform(1.1, 1.8)
        _, d = O.hllc(qL, qR, g)
        lhs = (d["ss"] - d["sL"]) * d["UsL"] + (d["sR"] - d["ss"]) * d["UsR"]
        rhs = d["sR"] * d["UR"] - d["sL"] * d["UL"] - (d["FR"] - d["FL"])
        scale = np.abs(rhs).max() + np.abs(d["sR"] * d["UR"]).max()
        assert np.abs(lhs - rhs).max() <= 1e-12 * scale


def test_paper_literal_energy_star_fails_consistency():
    """The energy entry of the star state exactly as printed breaks the consistency condition
    (the reason the standard Toro expression is used)."""
    rng = np.random.default_rng(4)
    worst = 0.0
    for _ in range(50):
        qL, qR, g = _rand_state(rng), _rand_state(rng), 1.4
        _, d = O.hllc(qL, qR, g, literal=True)
        lhs = (d["ss"] - d["sL"]) * d["UsL"] + (d["sR"] - d["ss"]) * d["UsR"]
        rhs = d["sR"] * d["UR"] - d["sL"] * d["UL"] - (d["FR"] - d["FL"])
        worst = max(worst, abs(lhs[3] - rhs[3]) / (abs(rhs[3]) + 1e-300))
        assert np.abs(lhs[:3] - rhs[:3]).max() <= 1e-11 * (np.abs(rhs).max() + 1)
    assert worst > 1e-3


def test_hllc_reduces_to_physical_flux_for_equal_states():
    rng = np.random.default_rng(5)
    for _ in range(100):
        q, g = _rand_state(rng), rng.uniform(1.1, 1.8)
        F, _ = O.hllc(q, q, g)
        Fp, _ = _phys_flux(q, g)
        assert np.abs(F - Fp).max() <= 1e-13 * (np.abs(Fp).max() + 1)


def test_hllc_upwinds_supersonic_states():
    g = 1.4
    qL = np.array([1.0, 5.0, 0.3, 1.0])   # sL = min(uL - aL, uR - aR) > 0
    qR = np.array([0.8, 4.0, -0.1, 0.7])
    F, d = O.hllc(qL, qR, g)
    assert d["sL"] > 0
    assert np.array_equal(F, d["FL"])
    qL2 = np.array([1.0, -5.0, 0.3, 1.0])
    qR2 = np.array([0.8, -4.0, -0.1, 0.7])
    F2, d2 = O.hllc(qL2, qR2, g)
    assert d2["sR"] < 0
    assert np.array_equal(F2, d2["FR"])


def test_hllc_preserves_stationary_contact():
    g = 1.4
    F, d = O.hllc(np.array([1.0, 0.0, 0.7, 2.0]), np.array([0.2, 0.0, -0.4, 2.0]), g)
    assert d["ss"] == 0.0
    assert np.array_equal(F, np.array([0.0, 2.0, 0.0, 0.0]))


def test_hllc_average_at_zero_contact_speed_is_the_star_pressure_flux():
    """At s* = 0 (reading O4: the average of both branches) with sL < 0 < sR, each branch's
    star flux F_K + s_K (U*_K - U_K) reduces to (0, p_K - m_K u_K, 0, 0), m_K = rho_K (s_K -
    u_K).  Symmetric collisions and expansions (normal velocities +w | -w, equal rho and p,
    different tangential velocities) give s* = 0 exactly with u != 0; the oracle's two-branch
    average must equal that closed form, which the fast GPU kernels evaluate instead of the
    branches.  Using F_K without the star correction (spm = 0), a sign slip in the star energy
    or star momentum, or the wrong wave speed in a branch breaks it."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        g = rng.uniform(1.1, 1.8)
        r, p, w = rng.uniform(0.2, 3.0), rng.uniform(0.2, 3.0), rng.uniform(-1.5, 1.5)
        qL = np.array([r, w, rng.uniform(-1, 1), p])
        qR = np.array([r, -w, rng.uniform(-1, 1), p])
        F, d = O.hllc(qL, qR, g)
        assert d["ss"] == 0.0 and d["sL"] < 0.0 < d["sR"]
        mL, mR = r * (d["sL"] - w), r * (d["sR"] + w)
        pstar = 0.5 * ((p - mL * w) + (p + mR * w))
        scale = p + r * (abs(w) + np.sqrt(g * p / r)) ** 2
        assert np.abs(F - np.array([0.0, pstar, 0.0, 0.0])).max() <= 1e-13 * scale


# ---------------------------------------------------------------------------------------
# solver-level invariants
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("mu,nu", [(0.0, 0.0), (2e-3, 0.0), (0.0, 1e-3), (1e-3, 5e-4)])
def test_conservation_on_periodic_domain(mu, nu):
    p = W.random_periodic(48, 40, seed=7, mu=mu, nu=nu)
    U0 = O.prim_to_cons(p, p.W0)
    dt = 0.5 * O.max_dt(p, U0, 0.5)
    U = O.step(p, U0, np.full(150, dt))
    s0, s1 = U0.sum(axis=(1, 2)), U.sum(axis=(1, 2))
    scale = np.abs(U0).sum(axis=(1, 2))
    assert (np.abs(s1 - s0) / scale).max() < 1e-13
    # and the state did change
    assert np.abs(U - U0).max() > 1e-3


def test_four_quadrant_problem_is_transpose_symmetric():
    p = W.riemann2d(64)
    U0 = O.prim_to_cons(p, p.W0)
    dts = [O.max_dt(p, U0, 0.5)] * 25
    U = O.step(p, U0, dts)
    UT = np.stack([U[0].T, U[2].T, U[1].T, U[3].T])
    assert np.array_equal(U, UT)


def test_two_d_with_uniform_rows_equals_one_d():
    p1 = W.sod(120)
    U1 = O.prim_to_cons(p1, p1.W0)
    ny = 8
    p2 = p1.with_(ny=ny, dy=1.0 / 120, bc=(0, 0, 2, 2), W0=np.repeat(p1.W0, ny, axis=1))
    U2 = O.prim_to_cons(p2, p2.W0)
    dts = [O.max_dt(p1, U1, 0.5)] * 40
    assert O.max_dt(p1, U1, 0.5) > 0
    A = O.step(p1, U1, dts)
    B = O.step(p2, U2, dts)
    for j in range(ny):
        assert np.array_equal(B[:, j], A[:, 0])


def test_viscous_terms_are_second_order_diffusion():
    """Shear layer u = u0 sin(2 pi y), rho = p = 1: the x-momentum RHS equals the exact
    viscous term mu d2u/dy2 to second order; the other components vanish to round-off."""
    errs = []
    for n in (32, 64, 128):
        p = W.random_periodic(8, n, seed=0).with_(dx=1.0 / n, dy=1.0 / n, mu=1e-2, Pr=0.72)
        y = (np.arange(n) + 0.5) / n
        Wp = np.zeros((4, n, 8))
        Wp[0] = 1.0
        Wp[3] = 1.0
        # cell averages of sin(2 pi y)
        avg = (np.cos(2 * np.pi * (y - 0.5 / n)) - np.cos(2 * np.pi * (y + 0.5 / n))) * n / (2 * np.pi)
        Wp[1] = avg[:, None]
        U = O.prim_to_cons(p, Wp)
        L = O.rhs(p, U)
        exact = -1e-2 * (2 * np.pi) ** 2 * avg
        errs.append(np.abs(L[1, :, 0] - exact).max())
        assert np.abs(L[0]).max() < 1e-12 and np.abs(L[2]).max() < 1e-12
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 1.9, orders


def _viscous_part(p, Wp, mu):
    """rhs(mu) - rhs(0): the inviscid terms do not depend on mu, so this is the viscous part."""
    U = O.prim_to_cons(p, Wp)
    return O.rhs(p.with_(mu=mu), U) - O.rhs(p.with_(mu=0.0), U)


@pytest.mark.parametrize("case", ["normal_stress_and_work", "heat_conduction", "shear_heating"])
def test_viscous_stress_work_and_heat_terms_converge_to_closed_forms(case):
    """The viscous part of the RHS against the Navier-Stokes terms it discretises (constant mu,
    Stokes hypothesis, kappa = mu gamma / ((gamma - 1) Pr), T = p / rho), second order:
    u = u0 sin(2 pi x): d(tau_xx)/dx = 4/3 mu u'', energy 4/3 mu (u'^2 + u u'');
    T = 1 + 0.1 sin(2 pi y) at rest, p = 1: energy kappa T'';
    u = u0 sin(2 pi y): energy mu (u'^2 + u u'')."""
    mu, g, Pr, u0 = 1e-2, 1.4, 0.72, 0.3
    kappa = mu * g / ((g - 1.0) * Pr)
    errs = []
    for n in (32, 64, 128):
        s = (np.arange(n) + 0.5) / n
        k = 2 * np.pi
        if case == "normal_stress_and_work":
            p = W.random_periodic(n, 8, seed=0).with_(dx=1.0 / n, dy=1.0 / n, Pr=Pr, gamma=g)
            Wp = np.zeros((4, 8, n))
            Wp[0], Wp[3] = 1.0, 1.0
            u = u0 * np.sin(k * s)
            Wp[1] = u[None, :]
            V = _viscous_part(p, Wp, mu)[:, 0, :]
            up, upp = u0 * k * np.cos(k * s), -u0 * k * k * np.sin(k * s)
            ex = {1: 4.0 / 3.0 * mu * upp, 3: 4.0 / 3.0 * mu * (up * up + u * upp)}
            assert np.abs(V[0]).max() < 1e-12 and np.abs(V[2]).max() < 1e-12
        elif case == "heat_conduction":
            p = W.random_periodic(8, n, seed=0).with_(dx=1.0 / n, dy=1.0 / n, Pr=Pr, gamma=g)
            Wp = np.zeros((4, n, 8))
            T = 1.0 + 0.1 * np.sin(k * s)
            Wp[0] = (1.0 / T)[:, None]
            Wp[3] = 1.0
            V = _viscous_part(p, Wp, mu)[:, :, 0]
            ex = {3: kappa * (-0.1 * k * k * np.sin(k * s))}
            assert np.abs(V[:3]).max() < 1e-12
        else:
            p = W.random_periodic(8, n, seed=0).with_(dx=1.0 / n, dy=1.0 / n, Pr=Pr, gamma=g)
            Wp = np.zeros((4, n, 8))
            Wp[0], Wp[3] = 1.0, 1.0
            u = u0 * np.sin(k * s)
            Wp[1] = u[:, None]
            V = _viscous_part(p, Wp, mu)[:, :, 0]
            up, upp = u0 * k * np.cos(k * s), -u0 * k * k * np.sin(k * s)
            ex = {1: mu * upp, 3: mu * (up * up + u * upp)}
        errs.append(max(np.abs(V[c] - e).max() / np.abs(e).max() for c, e in ex.items()))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 1.9 and errs[-1] < 5e-3, (errs, orders)


# ---------------------------------------------------------------------------------------
# immersed boundary (Sec. 2, Fig. 1(c)) and Rankine-Hugoniot initial states
# ---------------------------------------------------------------------------------------
def test_post_shock_state_matches_paper_mach5_state():
    g = golden("paper_mach5_post_shock.txt")[0]
    got = W.post_shock_state(g[0], g[1], g[2], g[3])
    assert np.allclose(got, g[4:8], rtol=1e-14, atol=1e-14)


def test_post_shock_derivatives_match_finite_differences():
    for M in (1.5, 2.0, 2.7):
        dM, dg = W.post_shock_state_derivs(M, 1.0, 1.0, 1.4)
        h = 1e-6
        fdM = (W.post_shock_state(M + h) - W.post_shock_state(M - h)) / (2 * h)
        fdg = (W.post_shock_state(M, gamma=1.4 + h) - W.post_shock_state(M, gamma=1.4 - h)) / (2 * h)
        assert np.allclose(dM, fdM, rtol=1e-7, atol=1e-9)
        assert np.allclose(dg, fdg, rtol=1e-7, atol=1e-9)


def _half_plane_problem(n=32, wall_row=10, u0=0.7):
    dx = 1.0 / n
    p = W.random_periodic(n, n, seed=0).with_(bc=(2, 2, 0, 0))
    X, Y = W.cell_centres(n, n, 0.0, 0.0, dx, dx)
    sdf = Y - wall_row * dx  # solid below the cell face y = wall_row * dx
    Wp = np.zeros((4, n, n))
    Wp[0] = 1.3
    Wp[1] = u0
    Wp[3] = 0.9
    return p.with_(sdf=sdf, W0=Wp)


def test_slip_wall_keeps_uniform_tangential_flow():
    p = _half_plane_problem()
    U = O.prim_to_cons(p, p.W0)
    L = O.rhs(p, U)
    assert np.abs(L).max() < 1e-13


def test_ib_tables_are_consistent():
    p = W.shock_cylinder(nx=128, ny=64)
    t = O.ib_tables(p)
    tag = t["tag"]
    assert (tag[p.sdf >= 0] == 0).all() and (tag[p.sdf < 0] > 0).all()
    assert np.allclose(t["w"].sum(axis=1), 1.0, atol=1e-14)
    flat = tag.reshape(-1)
    assert (flat[t["gcell"]] == 2).all()
    assert (flat[t["icell"]][t["w"] > 0] == 0).all()
    assert np.allclose(np.hypot(t["nrm"][:, 0], t["nrm"][:, 1]), 1.0, atol=1e-14)
    # every solid cell within three cells (box) of a fluid cell is a ghost
    ny, nx = tag.shape
    for j in range(ny):
        for i in range(nx):
            if tag[j, i] == 0:
                continue
            box = tag[max(0, j - 3):j + 4, max(0, i - 3):i + 4]
            assert (tag[j, i] == 2) == bool((box == 0).any())


def test_ib_wall_matches_reflective_boundary():
    """A cell-aligned immersed wall and a reflective domain boundary at the same place give
    the same fluid solution (to round-off)."""
    n, wall = 32, 8
    p_ib = _half_plane_problem(n, wall)
    Wp = W.random_state(p_ib, seed=3, amp=0.2)
    Wp[2] = 0.3 * np.sin(2 * np.pi * np.arange(n) / n)[None, :] * np.ones((n, 1))
    U_ib = O.prim_to_cons(p_ib, Wp)
    dx = 1.0 / n
    p_bc = p_ib.with_(ny=n - wall, y0=wall * dx, sdf=None, bc=(2, 2, 1, 0), W0=Wp[:, wall:])
    U_bc = O.prim_to_cons(p_bc, Wp[:, wall:])
    dts = [0.2 * O.max_dt(p_bc, U_bc, 0.5)] * 5
    A = O.step(p_ib, U_ib, dts)[:, wall:]
    B = O.step(p_bc, U_bc, dts)
    assert np.abs(A - B).max() < 1e-12 * np.abs(B).max()


# ---------------------------------------------------------------------------------------
# the oracle's forward-mode derivative against central finite differences
# ---------------------------------------------------------------------------------------
def test_tangent_matches_finite_differences():
    p = W.shock_cylinder(nx=48, ny=24, mach=2.0, Re=200.0)
    Wp = W.random_state(p, seed=1, amp=0.02)
    U0 = O.prim_to_cons(p, Wp)
    th = p.theta()
    dts = [0.5 * O.max_dt(p, U0, 0.5)] * 3
    rng = np.random.default_rng(0)
    dU = rng.standard_normal(U0.shape) * np.abs(U0) * 1e-2
    dth = np.zeros(20)
    dth[0], dth[1], dth[4:8] = 0.3, 1e-3, rng.standard_normal(4)
    _, tan = O.step_tangent(p, U0, dU, dth, dts)
    h = 1e-6
    Up = O.step(p, U0 + h * dU, dts, theta=th + h * dth)
    Um = O.step(p, U0 - h * dU, dts, theta=th - h * dth)
    fd = (Up - Um) / (2 * h)
    assert np.abs(fd - tan).max() <= 1e-6 * np.abs(tan).max()


def test_op_counts_are_plausible():
    p = W.riemann2d(32)
    U = O.prim_to_cons(p, p.W0)
    c = O.count_rhs(p, U)
    flops = c["add"] + c["mul"] + c["div"] + c["sqrt"]
    per_cell = flops / p.cells
    assert 800 < per_cell < 2500, c


# ---------------------------------------------------------------------------------------
# the immersed boundary on an oblique wall (Sec. 2, Fig. 1(c): ghost states mirror the flow at
# the image point so that the wall has no normal flux and keeps the tangential velocity)
# ---------------------------------------------------------------------------------------
THETA_WALL = np.pi / 6  # 30 degrees


def _oblique_wall_problem(n=64):
    """Solid below the line through (0.3, 0) at 30 degrees on [0,1]^2 (it leaves through the
    bottom and right sides, so every image point lies inside the domain); transmissive sides.
    Returns the problem, the unit normal into the fluid and the tangent."""
    dx = 1.0 / n
    t = np.array([np.cos(THETA_WALL), np.sin(THETA_WALL)])
    nrm = np.array([-np.sin(THETA_WALL), np.cos(THETA_WALL)])
    X, Y = W.cell_centres(n, n, 0.0, 0.0, dx, dx)
    sdf = (X - 0.3) * nrm[0] + Y * nrm[1]  # exact signed distance to the line
    p = W.riemann2d(n).with_(sdf=sdf, bc=(0, 0, 0, 0))
    return p, nrm, t


def _garbage_in_solid(p, Wp):
    """Solid cells hold an unrelated state: the ghost fill, not the initial data, must give
    the wall its values."""
    solid = p.sdf < 0
    for c, v in enumerate((5.0, -3.0, 2.0, 7.0)):
        Wp[c][solid] = v
    return Wp


def test_oblique_slip_wall_keeps_uniform_tangential_flow():
    """Uniform flow parallel to a 30-degree wall is an exact steady solution: the mirrored
    ghosts reproduce it, so the RHS vanishes to round-off.  Fails if ghosts are not filled
    (garbage in the solid), for a no-slip mirror, or for a mirror that flips the tangential
    component."""
    p, nrm, t = _oblique_wall_problem()
    Wp = np.zeros((4, p.ny, p.nx))
    Wp[0], Wp[1], Wp[2], Wp[3] = 1.3, 0.7 * t[0], 0.7 * t[1], 0.9
    U = O.prim_to_cons(p, _garbage_in_solid(p, Wp))
    L = O.rhs(p, U)
    assert O.ib_tables(p)["gcell"].size > 100
    assert np.abs(L).max() < 1e-11  # fluxes O(1), 1/dx = 64


def _linear_prims(X, Y):
    return np.stack([1.0 + 0.3 * X + 0.2 * Y, 0.4 - 0.5 * X + 0.3 * Y, -0.2 + 0.6 * X - 0.1 * Y,
                     1.0 + 0.2 * X - 0.4 * Y])


def _ghost_cells(sdf):
    """Solid cells with a fluid cell in their 7x7 box (reading O7), computed here directly."""
    ny, nx = sdf.shape
    out = []
    for j in range(ny):
        for i in range(nx):
            if sdf[j, i] >= 0:
                continue
            box = sdf[max(0, j - 3):j + 4, max(0, i - 3):i + 4]
            if (box >= 0).any():
                out.append((j, i))
    return out


def _prims_of(U, gamma=1.4):
    r = U[0]
    u, v = U[1] / r, U[2] / r
    return np.stack([r, u, v, (gamma - 1.0) * (U[3] - 0.5 * r * (u * u + v * v))])


def test_oblique_slip_wall_ghosts_mirror_a_linear_field_at_the_image_point():
    """Ghost state = the slip-wall mirror (rho, p kept, V - 2 (V.n) n) of the interpolated
    primitive state at the image point x_G - 2 sdf_G n, computed here from the exact geometry.
    Bilinear interpolation reproduces a linear field exactly, so where the 2x2 interpolation
    block is all fluid the ghost equals the mirrored linear field at the image point; elsewhere
    it equals the bilinear weights restricted to fluid cells and renormalised (reading O7),
    written out here.  Fails for a wrong image-point distance (x_G - sdf n), a mirror of the
    wrong sign, swapped x/y weights or an inward normal."""
    p, nrm, _ = _oblique_wall_problem()
    n, dx = p.nx, p.dx
    X, Y = W.cell_centres(n, n, 0.0, 0.0, dx, dx)
    Wp = _garbage_in_solid(p, _linear_prims(X, Y))
    U = O.prim_to_cons(p, Wp)
    out = O.ib_fill(p, U)
    ghosts = _ghost_cells(p.sdf)
    changed = np.argwhere((out != U).any(axis=0))
    assert sorted(map(tuple, changed)) == sorted(ghosts)
    Q = _prims_of(out)
    Qf = _prims_of(U)
    exact_checked = 0
    for j, i in ghosts:
        xg, yg = X[j, i], Y[j, i]
        phi = p.sdf[j, i]
        xi, yi = xg - 2.0 * phi * nrm[0], yg - 2.0 * phi * nrm[1]
        fx, fy = xi / dx - 0.5, yi / dx - 0.5
        i0 = min(max(int(np.floor(fx)), 0), n - 2)
        j0 = min(max(int(np.floor(fy)), 0), n - 2)
        tx, ty = fx - i0, fy - j0
        cells = [(j0, i0), (j0, i0 + 1), (j0 + 1, i0), (j0 + 1, i0 + 1)]
        w = np.array([(1 - tx) * (1 - ty), tx * (1 - ty), (1 - tx) * ty, tx * ty])
        fluid = np.array([p.sdf[c] >= 0 for c in cells])
        w = np.where(fluid, w, 0.0)
        w = w / w.sum()
        q = sum(w[k] * Qf[:, cells[k][0], cells[k][1]] for k in range(4))
        if fluid.all():
            q_lin = _linear_prims(np.array(xi), np.array(yi))
            assert np.abs(q - q_lin).max() < 1e-13
            q = q_lin
            exact_checked += 1
        V = q[1:3]
        Vg = V - 2.0 * (V @ nrm) * nrm
        want = np.array([q[0], Vg[0], Vg[1], q[3]])
        assert np.abs(Q[:, j, i] - want).max() < 1e-12, (j, i, Q[:, j, i], want)
    assert exact_checked > 50


# ---------------------------------------------------------------------------------------
# the positivity fallback (reading O6 of "positivity-preserving HLLC", Sec. 2)
# ---------------------------------------------------------------------------------------
def _rough_1d(n=200, seed=0):
    rng = np.random.default_rng(seed)
    p = W.sod(n).with_(name="rough")
    Wp = np.zeros((4, 1, n))
    Wp[0, 0] = 10 ** rng.uniform(-2, 1, n)
    Wp[1, 0] = rng.uniform(-1, 1, n)
    Wp[2, 0] = rng.uniform(-0.5, 0.5, n)
    Wp[3, 0] = 10 ** rng.uniform(-4, 2, n)
    return p, Wp


@pytest.mark.parametrize("seed", [0, 1])
def test_positivity_fallback_uses_first_order_states_exactly_where_weno_fails(seed):
    """On a rough 1D state (density over 3 and pressure over 6 decades) WENO5 reconstructs a
    non-positive density or pressure at many faces.  The RHS must equal the flux divergence
    built here from the pinned building blocks: at faces where a reconstructed rho or p is
    <= 0, HLLC of the two adjacent CELL states; elsewhere HLLC of the WENO5 states.  The
    oracle's count of fallback faces must equal the count found here.  Fails if the fallback is
    skipped, tests only rho, or takes other cells' states."""
    p, Wp = _rough_1d(seed=seed)
    n = p.nx
    U = O.prim_to_cons(p, Wp)
    q = _prims_of(U[:, 0, :])
    qp = np.concatenate([np.repeat(q[:, :1], 3, axis=1), q, np.repeat(q[:, -1:], 3, axis=1)], axis=1)
    F = np.zeros((4, n + 1))
    fallbacks = 0
    for f in range(n + 1):
        il, ir = f + 2, f + 3  # padded indices of the cells left and right of face f
        qL = np.array([O.weno5(qp[c, il - 2:il + 3]) for c in range(4)])
        qR = np.array([O.weno5(qp[c, ir - 2:ir + 3][::-1]) for c in range(4)])
        if not (qL[0] > 0 and qL[3] > 0 and qR[0] > 0 and qR[3] > 0):
            qL, qR = qp[:, il], qp[:, ir]
            fallbacks += 1
        F[:, f], _ = O.hllc(qL, qR, p.gamma)
    want = -(F[:, 1:] - F[:, :-1]) / p.dx
    O.fallback_faces()
    L = O.rhs(p, U)[:, 0, :]
    assert O.fallback_faces() == fallbacks and fallbacks > 20
    assert np.abs(L - want).max() <= 1e-12 * np.abs(want).max()


def test_positivity_fallback_occurs_in_the_blast_wave_problem():
    """The two interacting blast waves (pressures 1000 | 0.01 | 100, reflective ends): the
    fallback is first taken at step 942 (t = 0.02706), at two faces, and the run stays
    physical through it."""
    n = 400
    p = W.sod(n).with_(name="blast", bc=(1, 1, 0, 0))
    x = (np.arange(n) + 0.5) / n
    Wp = np.zeros((4, 1, n))
    Wp[0] = 1.0
    Wp[3, 0] = np.where(x < 0.1, 1000.0, np.where(x < 0.9, 0.01, 100.0))
    U = O.prim_to_cons(p, Wp)
    O.fallback_faces()
    first = None
    for k in range(1, 960):
        U = O.step(p, U, [O.max_dt(p, U, 0.5)])
        c = O.fallback_faces()
        if c and first is None:
            first = (k, c)
    assert first == (942, 2)
    assert U[0].min() > 0 and _prims_of(U[:, 0, :])[3].min() > 0


# ---------------------------------------------------------------------------------------
# the CFL rule (reading O2), from values worked out by hand
# ---------------------------------------------------------------------------------------
def _cfl_problem(mu, Pr):
    """A 6 x 6 grid (dx = 0.1, dy = 0.2, gamma = 1.4) tiled with three states whose sound
    speeds are whole numbers: (rho, u, v, a) = (1, 0.5, -0.25, 1), (4, -2, 0, 0.5),
    (0.25, 0, 1, 2), p = rho a^2 / 1.4 = 1/1.4 for all three.  Their rates
    (|u| + a)/dx + (|v| + a)/dy are 15 + 6.25 = 21.25, 25 + 2.5 = 27.5 and 20 + 15 = 35.
    A solid cell (sdf < 0) holds a state with a rate of 10^4 that must not count."""
    states = [(1.0, 0.5, -0.25, 1.0 / 1.4), (4.0, -2.0, 0.0, 1.0 / 1.4), (0.25, 0.0, 1.0, 1.0 / 1.4)]
    Wp = np.zeros((4, 6, 6))
    for j in range(6):
        for i in range(6):
            Wp[:, j, i] = states[(i + j) % 3]
    Wp[:, 2, 3] = (1.0, 1000.0, 0.0, 1.0)
    X, Y = W.cell_centres(6, 6, 0.0, 0.0, 0.1, 0.2)
    sdf = np.hypot(X - (0.35 + 0.01), Y - (0.5 + 0.02)) - 0.05  # a small body: cell (2, 3) alone is solid
    assert (sdf < 0).sum() == 1 and sdf[2, 3] < 0
    p = W.Problem("cfl", 6, 6, 0.0, 0.0, 0.1, 0.2, bc=(0, 0, 0, 0), mu=mu, Pr=Pr, sdf=sdf, W0=Wp)
    return p


@pytest.mark.parametrize("mu,Pr,want", [
    (0.0, 0.72, 0.5 / 35.0),                                      # convective limit
    (1e-3, 0.72, 0.5 / 35.0),                                     # viscous cap above it
    (0.1, 0.72, 0.5 * 0.1 * 0.1 * 0.25 / (2 * 0.1 * (1.4 / 0.72))),  # cap: gamma/Pr > 4/3
    (0.1, 2.0, 0.5 * 0.1 * 0.1 * 0.25 / (2 * 0.1 * (4.0 / 3.0))),    # cap: 4/3 > gamma/Pr
])
def test_cfl_step_matches_hand_computed_values(mu, Pr, want):
    """dt = CFL / 35 from the fastest fluid state, or the viscous cap
    CFL h^2 rho_min / (2 mu max(4/3, gamma/Pr)) with h = min(dx, dy) = 0.1, rho_min = 0.25,
    when that is smaller.  Fails for a wrong max/min, h = max(dx, dy), a missing viscous
    factor or a solid cell counted."""
    p = _cfl_problem(mu, Pr)
    U = O.prim_to_cons(p, p.W0)
    assert O.max_dt(p, U, 0.5) == pytest.approx(want, rel=1e-14)
