"""Writes the oracle's reference runs of the two full-size benchmark configurations at their
full step counts, for the GPU parity tests that cannot run the oracle themselves (it needs CPU
hours for these):

  fullrun_shock_cylinder_2048x1024.txt  viscous Mach-2 shock over the immersed cylinder,
                                        2048 x 1024 cells, 2000 CFL steps (CFL 0.5)
  fullrun_riemann2d_1024.txt            four-quadrant Riemann problem, 1024 x 1024 cells,
                                        CFL 0.5 to t = 0.8 (last step clipped)

Each run starts from the oracle's conserved form of the workload's primitive initial state and
takes, step after step, the oracle's CFL step of the current state (the last one clipped to the
end time: dt = t_end - t when t + dt > t_end, t accumulated as t = t + dt), then one oracle
SSP-RK3 step.  At each checkpoint the file records the step count, the time, SHA-256 digests of
the state's float64 bytes ([4][ny][nx], little-endian) and of the step sizes so far, the
normwise scales (max |rho|, max |momentum vector|, max |E|) and sampled cells: half of them
seeded uniform over the grid, half seeded among the cells of steepest density change (where
differences between implementations concentrate).  Values are written with repr(), which
round-trips float64 exactly.  Calls only oracle/ and the input generators.

    python tests/golden/make_fullrun_goldens.py [shock_cylinder|riemann2d ...]
"""
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2601_04400_gb300 import workloads as W  # noqa: E402

NSAMPLE = 512  # per half, per checkpoint

CASES = {
    "shock_cylinder": dict(make=lambda: W.shock_cylinder(), checkpoints=(1000, 2000),
                           out="fullrun_shock_cylinder_2048x1024.txt"),
    "riemann2d": dict(make=lambda: W.riemann2d(1024), checkpoints=(1000, None),
                      out="fullrun_riemann2d_1024.txt"),
}


def sha256(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<f8").tobytes()).hexdigest()


def scales(U):
    return (float(np.abs(U[0]).max()), float(np.sqrt(U[1] ** 2 + U[2] ** 2).max()), float(np.abs(U[3]).max()))


def sample_cells(U, k):
    ny, nx = U.shape[1:]
    rng = np.random.default_rng(1000 + k)
    uni = rng.choice(nx * ny, NSAMPLE, replace=False)
    r = U[0]
    g = np.zeros_like(r)
    g[1:-1, :] += np.abs(r[2:, :] - r[:-2, :])
    g[:, 1:-1] += np.abs(r[:, 2:] - r[:, :-2])
    flat = g.reshape(-1)
    steep = np.argsort(flat)[-(nx * ny) // 50:]  # the steepest 2%
    steep = rng.choice(steep, NSAMPLE, replace=False)
    cells = np.unique(np.concatenate([uni, steep]))
    return [(int(c // nx), int(c % nx)) for c in cells]


def run(name):
    spec = CASES[name]
    p = spec["make"]()
    U = O.prim_to_cons(p, p.W0)
    t_end = p.t_end
    max_steps = p.n_steps if p.n_steps is not None else 10 ** 9
    lines = ["# Oracle reference run: %s %dx%d, CFL %g, %s (written by make_fullrun_goldens.py; oracle only)"
             % (name, p.nx, p.ny, p.cfl, ("t_end %r" % t_end) if t_end is not None else "%d steps" % max_steps),
             "case %s nx %d ny %d cfl %r" % (name, p.nx, p.ny, p.cfl)]
    t, dts, k = 0.0, [], 0
    t0 = time.time()
    wanted = set(c for c in spec["checkpoints"] if c is not None)

    def checkpoint():
        s = scales(U)
        lines.append("checkpoint %d t %r state_sha256 %s dts_sha256 %s scale %r %r %r"
                     % (k, t, sha256(U), sha256(np.array(dts)), s[0], s[1], s[2]))
        for j, i in sample_cells(U, k):
            lines.append("sample %d %d %d %r %r %r %r" % ((k, j, i) + tuple(float(U[c, j, i]) for c in range(4))))
        print("%s: checkpoint at step %d, t = %.6f (%.0f s)" % (name, k, t, time.time() - t0), flush=True)

    while k < max_steps and (t_end is None or t < t_end):
        dt = O.max_dt(p, U, p.cfl)
        if t_end is not None and t + dt > t_end:
            dt = t_end - t
        U = O.step(p, U, [dt])
        t = t + dt
        dts.append(dt)
        k += 1
        if k in wanted:
            checkpoint()
        if k % 100 == 0:
            print("%s: step %d t %.6f (%.0f s)" % (name, k, t, time.time() - t0), flush=True)
    if k not in wanted:
        checkpoint()
    lines.append("steps %d" % k)
    with open(os.path.join(HERE, spec["out"]), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    for name in (sys.argv[1:] or list(CASES)):
        run(name)
