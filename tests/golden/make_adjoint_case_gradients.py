"""Writes adjoint_case_512_gradients.txt: the exact discrete derivatives, by the oracle's forward
mode, of the adjoint workload's loss (the viscous shock-cylinder case of Sec. 3 scaled to
[0, 4D]^2 at 512 x 512 cells, Re = 1000 at Mach 2 with mu held at 3.9443e-3, 400 SSP-RK3 steps
of the fixed dt given by CFL 0.5 on the Mach-2.2 initial state):

    L = sum over fluid cells of (rho - rho_target)^2 dx dy,  rho_target = the Mach-2.2 run,

with respect to the shock Mach number (through the initial post-shock state and the inflow
state: the Rankine-Hugoniot derivatives of the input generator), gamma (the solver parameter,
the initial conserved energy p/(gamma - 1) and the post-shock state) and mu, at Mach 2, gamma
1.4.  Calls only oracle/ and the input generators (about 12 CPU-minutes).

    python tests/golden/make_adjoint_case_gradients.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2601_04400_gb300 import workloads as W  # noqa: E402

N, STEPS, MU0, MACH, GAMMA = 512, 400, 3.9443e-3, 2.0, 1.4


def problem(M, gamma=GAMMA):
    return W.adjoint_case(N, mach=M, gamma=gamma, n_steps=STEPS).with_(mu=MU0)


def cons(W0, gamma):
    r, u, v, p = W0
    return np.stack([r, r * u, r * v, p / (gamma - 1.0) + 0.5 * r * (u * u + v * v)])


def cons_tangent(W0, dW):
    """Tangent of the conserved state for a tangent dW of the primitive state (gamma fixed)."""
    r, u, v, _ = W0
    return np.stack([dW[0], dW[0] * u + r * dW[1], dW[0] * v + r * dW[2],
                     dW[0] * 0.5 * (u * u + v * v) + r * (u * dW[1] + v * dW[2]) + dW[3] / (GAMMA - 1.0)])


def main():
    pt = problem(2.2)
    Ut0 = cons(pt.W0, GAMMA)
    dt = O.max_dt(pt, Ut0, 0.5)
    rho_t = O.step(pt, Ut0, [dt] * STEPS)[0]
    p = problem(MACH)
    U0 = cons(p.W0, GAMMA)
    fluid = O.ib_tables(p)["tag"] == 0
    dWdM, dWdg = W.post_shock_state_derivs(MACH, 1.0, 1.0, GAMMA)
    behind = (W.cell_centres(p.nx, p.ny, 0.0, 0.0, p.dx, p.dy)[0] < p.meta["x_shock"]).astype(float)
    dirs = {}
    # Mach: the post-shock initial state and the x-low inflow state (parameters 4..7)
    dth = np.zeros(20)
    dth[4:8] = dWdM
    dirs["mach"] = (cons_tangent(p.W0, behind[None] * np.asarray(dWdM)[:, None, None]), dth)
    # gamma: the parameter, the post-shock state, the inflow state and E = p / (gamma - 1) + ...
    dth = np.zeros(20)
    dth[0] = 1.0
    dth[4:8] = dWdg
    dU = cons_tangent(p.W0, behind[None] * np.asarray(dWdg)[:, None, None])
    dU[3] += -p.W0[3] / (GAMMA - 1.0) ** 2
    dirs["gamma"] = (dU, dth)
    # mu
    dth = np.zeros(20)
    dth[1] = 1.0
    dirs["mu"] = (np.zeros_like(U0), dth)
    out = {}
    for name, (dU0, dth) in dirs.items():
        UN, dUN = O.step_tangent(p, U0, dU0, dth, [dt] * STEPS)
        d = (UN[0] - rho_t) * fluid
        out["L"] = float((d * d).sum()) * p.dx * p.dy
        out[name] = float((2.0 * d * dUN[0]).sum()) * p.dx * p.dy
        print(name, repr(out[name]), flush=True)
    path = os.path.join(HERE, "adjoint_case_512_gradients.txt")
    with open(path, "w") as f:
        f.write("# Exact discrete derivatives of the adjoint workload's loss (512^2, 400 steps, Mach 2,\n")
        f.write("# gamma 1.4, mu 3.9443e-3, dt from CFL 0.5 on the Mach-2.2 state): oracle forward mode.\n")
        f.write("# Written by tests/golden/make_adjoint_case_gradients.py.  Columns: dt L dL/dMach dL/dgamma dL/dmu\n")
        f.write("%r %r %r %r %r\n" % (dt, out["L"], out["mach"], out["gamma"], out["mu"]))
    print(path)


if __name__ == "__main__":
    main()
