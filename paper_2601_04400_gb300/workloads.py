"""Seeded synthetic workloads shaped like the paper's test cases.

This module only builds inputs: grids, boundary kinds, parameters, signed-distance fields of
the immersed solid and PRIMITIVE initial states (rho, u, v, p).  It holds none of the
solver's arithmetic (no EOS, no fluxes), so that both the CUDA path and the CPU oracle can
take their inputs from it.  Each side converts primitives to conserved variables with its
own code.

Cases (Sec. 3 of the paper, sizes of the throughput and parity workloads):
  * ``sod``            1D Sod shock tube, (rho, u, p) = (1, 0, 1) | (0.125, 0, 0.1), x = 0.5.
  * ``riemann2d``      2D four-quadrant Riemann problem on [0,1]^2 split at (0.8, 0.8).
  * ``shock_cylinder`` viscous planar shock (Rankine-Hugoniot post-shock state) over an
                       immersed circular cylinder, reflective top/bottom, inflow left.
  * ``adjoint_case``   the shock-cylinder case scaled to [0,4D]^2 for the adjoint.
  * ``batched_cases``  many shock-cylinder instances with seeded Mach, radius and grids.
  * ``smooth_wave``    periodic density wave for convergence-order checks.
  * ``random_periodic`` smooth random periodic states for conservation checks.
"""
from dataclasses import dataclass, field, replace
from typing import Optional, Tuple

import numpy as np

BC_TRANSMISSIVE, BC_REFLECTIVE, BC_PERIODIC, BC_INFLOW = 0, 1, 2, 3


@dataclass
class Problem:
    name: str
    nx: int
    ny: int
    x0: float
    y0: float
    dx: float
    dy: float
    bc: Tuple[int, int, int, int] = (0, 0, 0, 0)
    gamma: float = 1.4
    mu: float = 0.0
    Pr: float = 0.72
    nu: float = 0.0
    inflow: np.ndarray = field(default_factory=lambda: np.tile([1.0, 0.0, 0.0, 1.0], (4, 1)))
    wall: int = 0
    sdf: Optional[np.ndarray] = None
    W0: Optional[np.ndarray] = None    # primitive initial state [4, ny, nx]
    cfl: float = 0.5
    t_end: Optional[float] = None
    n_steps: Optional[int] = None
    meta: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def theta(self) -> np.ndarray:
        """Parameter vector [gamma, mu, Pr, nu, inflow(4 sides x rho,u,v,p)]."""
        th = np.zeros(20)
        th[:4] = (self.gamma, self.mu, self.Pr, self.nu)
        th[4:] = np.asarray(self.inflow, dtype=np.float64).reshape(16)
        return th

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


def cell_centres(nx, ny, x0, y0, dx, dy):
    x = x0 + (np.arange(nx) + 0.5) * dx
    y = y0 + (np.arange(ny) + 0.5) * dy
    return np.meshgrid(x, y)  # [ny, nx] each


# ---------------------------------------------------------------------------------------
# Rankine-Hugoniot post-shock state of a normal shock of Mach M moving into gas at rest
# (initial condition of the shock-cylinder cases; the paper's Mach-5 state {7, 4, 0, 29}
# into (rho, p) = (1.4, 1) is reproduced exactly).
# ---------------------------------------------------------------------------------------
def post_shock_state(M, rho1=1.0, p1=1.0, gamma=1.4):
    a1 = np.sqrt(gamma * p1 / rho1)
    rho2 = rho1 * (gamma + 1.0) * M * M / ((gamma - 1.0) * M * M + 2.0)
    p2 = p1 * (2.0 * gamma * M * M - (gamma - 1.0)) / (gamma + 1.0)
    u2 = 2.0 * a1 / (gamma + 1.0) * (M - 1.0 / M)
    return np.array([rho2, u2, 0.0, p2])


def post_shock_state_derivs(M, rho1=1.0, p1=1.0, gamma=1.4):
    """d(rho2, u2, v2, p2)/dM and d(...)/dgamma of ``post_shock_state`` (analytic)."""
    a1 = np.sqrt(gamma * p1 / rho1)
    g1, g2 = gamma + 1.0, gamma - 1.0
    den = g2 * M * M + 2.0
    drho_dM = rho1 * g1 * (2.0 * M * den - M * M * 2.0 * g2 * M) / den ** 2
    dp_dM = p1 * 4.0 * gamma * M / g1
    du_dM = 2.0 * a1 / g1 * (1.0 + 1.0 / (M * M))
    dM = np.array([drho_dM, du_dM, 0.0, dp_dM])
    da1_dg = 0.5 * a1 / gamma
    drho_dg = rho1 * M * M * (den - g1 * M * M) / den ** 2
    dp_dg = p1 * ((2.0 * M * M - 1.0) * g1 - (2.0 * gamma * M * M - g2)) / g1 ** 2
    du_dg = 2.0 * (M - 1.0 / M) * (da1_dg * g1 - a1) / g1 ** 2
    dg = np.array([drho_dg, du_dg, 0.0, dp_dg])
    return dM, dg


# ---------------------------------------------------------------------------------------
# cases
# ---------------------------------------------------------------------------------------
def sod(n=200, t_end=0.2, cfl=0.5):
    """1D Sod shock tube (Sec. 3): transmissive ends, interface at x = 0.5."""
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    W = np.zeros((4, 1, n))
    left = x < 0.5
    W[0, 0] = np.where(left, 1.0, 0.125)
    W[3, 0] = np.where(left, 1.0, 0.1)
    return Problem("sod", n, 1, 0.0, 0.0, dx, 1.0, bc=(0, 0, 0, 0), W0=W, cfl=cfl, t_end=t_end,
                   meta=dict(left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1), x_disc=0.5))


def riemann2d(n=1024, t_end=0.8, cfl=0.5, split=0.8, ny=None):
    """2D four-quadrant Riemann problem on [0,1]^2, transmissive boundaries (n x ny cells)."""
    nx = n
    ny = n if ny is None else ny
    dx, dy = 1.0 / nx, 1.0 / ny
    X, Y = cell_centres(nx, ny, 0.0, 0.0, dx, dy)
    W = np.zeros((4, ny, nx))
    ne = (X >= split) & (Y >= split)
    nw = (X < split) & (Y >= split)
    sw = (X < split) & (Y < split)
    se = (X >= split) & (Y < split)
    for mask, st in ((ne, (1.5, 0.0, 0.0, 1.5)), (nw, (0.5323, 1.206, 0.0, 0.3)),
                     (sw, (0.138, 1.206, 1.206, 0.029)), (se, (0.5323, 0.0, 1.206, 0.3))):
        for c in range(4):
            W[c][mask] = st[c]
    return Problem("riemann2d", nx, ny, 0.0, 0.0, dx, dy, bc=(0, 0, 0, 0), W0=W, cfl=cfl, t_end=t_end)


def shock_cylinder(nx=2048, ny=1024, mach=2.0, Re=1000.0, Pr=0.72, gamma=1.4, D=1.0,
                   Lx=8.0, Ly=4.0, centre=(2.0, 2.0), radius=None, x_shock=1.0, n_steps=2000,
                   cfl=0.5, viscous=True):
    """Planar shock of Mach `mach` into quiescent gas (rho, p) = (1, 1) over a cylinder.

    Left boundary: inflow at the post-shock state; right: transmissive; top and bottom:
    reflective walls.  mu = rho2 u2 D / Re from the post-shock state.
    """
    r = 0.5 * D if radius is None else radius
    dx, dy = Lx / nx, Ly / ny
    X, Y = cell_centres(nx, ny, 0.0, 0.0, dx, dy)
    post = post_shock_state(mach, 1.0, 1.0, gamma)
    pre = np.array([1.0, 0.0, 0.0, 1.0])
    W = np.zeros((4, ny, nx))
    behind = X < x_shock
    for c in range(4):
        W[c] = np.where(behind, post[c], pre[c])
    sdf = np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2) - r
    mu = post[0] * post[1] * D / Re if viscous else 0.0
    inflow = np.array([post, pre, pre, pre])
    return Problem("shock_cylinder", nx, ny, 0.0, 0.0, dx, dy,
                   bc=(BC_INFLOW, BC_TRANSMISSIVE, BC_REFLECTIVE, BC_REFLECTIVE), gamma=gamma, mu=mu,
                   Pr=Pr, inflow=inflow, sdf=sdf, W0=W, cfl=cfl, n_steps=n_steps,
                   meta=dict(mach=mach, Re=Re, D=D, radius=r, centre=centre, x_shock=x_shock))


def mach5_cylinder(nx=4347, ny=1932, t_end=1.2, cfl=0.5):
    """The paper's shock-cylinder case (Sec. 3): (x, y) in [-0.5, 4] x [0, 2], cylinder of
    radius 0.25 at (0.6, 1), Euler, gamma = 1.4; (rho, u, v, p) = (7, 4, 0, 29) for x < 0.3
    (a Mach-5 shock moving into the gas at rest) and (1.4, 0, 0, 1) beyond; left inflow at the
    left state, right outflow (transmissive), reflective top and bottom.  The default grid has
    8.40e6 nearly square cells (the paper's uniform grid of about 8.4e6 cells)."""
    x0, y0, Lx, Ly = -0.5, 0.0, 4.5, 2.0
    dx, dy = Lx / nx, Ly / ny
    X, Y = cell_centres(nx, ny, x0, y0, dx, dy)
    left = np.array([7.0, 4.0, 0.0, 29.0])
    right = np.array([1.4, 0.0, 0.0, 1.0])
    W = np.zeros((4, ny, nx))
    behind = X < 0.3
    for c in range(4):
        W[c] = np.where(behind, left[c], right[c])
    sdf = np.sqrt((X - 0.6) ** 2 + (Y - 1.0) ** 2) - 0.25
    inflow = np.array([left, right, right, right])
    return Problem("mach5_cylinder", nx, ny, x0, y0, dx, dy,
                   bc=(BC_INFLOW, BC_TRANSMISSIVE, BC_REFLECTIVE, BC_REFLECTIVE), gamma=1.4, mu=0.0,
                   inflow=inflow, sdf=sdf, W0=W, cfl=cfl, t_end=t_end,
                   meta=dict(radius=0.25, centre=(0.6, 1.0), x_shock=0.3))


def adjoint_case(n=512, mach=2.0, n_steps=400, Re=1000.0, gamma=1.4):
    """Shock-cylinder case scaled to [0,4D]^2, cylinder r = D/2 at (2D, 2D), shock at x = D."""
    return shock_cylinder(nx=n, ny=n, mach=mach, Re=Re, gamma=gamma, Lx=4.0, Ly=4.0, n_steps=n_steps)


def batched_cases(count=256, seed=0, n_steps=500, mach_range=(1.5, 3.0), r_range=(0.3, 0.7),
                  nx_choices=tuple(range(128, 513, 64)), ny_choices=(128, 192, 256)):
    """Independent shock-cylinder instances with seeded Mach number, radius and grid."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nx = int(rng.choice(nx_choices))
        ny = int(rng.choice(ny_choices))
        mach = float(rng.uniform(*mach_range))
        r = float(rng.uniform(*r_range))
        p = shock_cylinder(nx=nx, ny=ny, mach=mach, radius=r, n_steps=n_steps)
        p.name = "batched_%d" % k
        out.append(p)
    return out


def smooth_wave(n, amp=0.2, t_end=0.1, cfl=0.5):
    """Periodic density wave rho = 1 + amp sin(2 pi x), u = 1, p = 1 on [0,1] (1D)."""
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    W = np.zeros((4, 1, n))
    # cell averages of the density wave
    W[0, 0] = 1.0 + amp * (np.cos(2 * np.pi * (x - 0.5 * dx)) - np.cos(2 * np.pi * (x + 0.5 * dx))) / (2 * np.pi * dx)
    W[1, 0] = 1.0
    W[3, 0] = 1.0
    return Problem("smooth_wave", n, 1, 0.0, 0.0, dx, 1.0, bc=(2, 2, 2, 2), W0=W, cfl=cfl, t_end=t_end,
                   meta=dict(amp=amp))


def random_periodic(nx, ny, seed=0, amp=0.3, modes=3, mu=0.0, nu=0.0):
    """Smooth random periodic state on [0,1]x[0,ny/nx] (all boundaries periodic)."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / nx
    X, Y = cell_centres(nx, ny, 0.0, 0.0, dx, dx)
    Ly = ny * dx
    W = np.zeros((4, ny, nx))
    base = (1.0, 0.3, -0.2, 1.0)
    for c in range(4):
        f = np.full((ny, nx), base[c])
        for _ in range(modes):
            kx, ky = rng.integers(1, 4), rng.integers(0, 3)
            ph = rng.uniform(0, 2 * np.pi)
            a = amp * rng.uniform(0.2, 1.0) * (0.5 if c in (0, 3) else 1.0)
            f = f + a * np.sin(2 * np.pi * (kx * X + ky * Y / Ly) + ph)
        W[c] = f
    return Problem("random_periodic", nx, ny, 0.0, 0.0, dx, dx, bc=(2, 2, 2, 2), mu=mu, nu=nu, W0=W)


def random_state(prob, seed=0, amp=0.05):
    """Seeded perturbation of a problem's primitive initial state (positive rho and p)."""
    rng = np.random.default_rng(seed)
    W = np.array(prob.W0, copy=True)
    W[0] *= 1.0 + amp * rng.uniform(-1, 1, W[0].shape)
    W[1] += amp * rng.uniform(-1, 1, W[1].shape)
    if prob.ny > 1:
        W[2] += amp * rng.uniform(-1, 1, W[2].shape)
    W[3] *= 1.0 + amp * rng.uniform(-1, 1, W[3].shape)
    return W


def uniform_normal(shape, seed=0):
    """Seeded standard-normal array (cotangents, tangents)."""
    return np.random.default_rng(seed).standard_normal(shape)
