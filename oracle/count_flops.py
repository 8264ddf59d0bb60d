"""Algorithmic FP64 operation count of one right-hand-side evaluation per cell, taken with
the oracle's counting scalar (one count per add/sub, mul, div and sqrt of the plain
formulation; every face evaluated once).  These are the per-unit figures of the roofline:
one SSP-RK3 step = 3 evaluations.

    python oracle/count_flops.py   -> prints a JSON line per workload
"""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle as O  # noqa: E402
from paper_2601_04400_gb300 import workloads as W  # noqa: E402


def count(prob, seed=0, amp=0.01):
    """Count on a seeded small perturbation of the workload's initial state, so that no face
    sees an exactly zero contact speed (where sign(s*) = 0 evaluates both HLLC branches)."""
    c = O.count_rhs(prob, O.prim_to_cons(prob, W.random_state(prob, seed=seed, amp=amp)))
    flops = c["add"] + c["mul"] + c["div"] + c["sqrt"]
    return dict(workload=prob.name, nx=prob.nx, ny=prob.ny, flops_per_cell_stage=flops / prob.cells,
                **{k + "_per_cell_stage": v / prob.cells for k, v in c.items()})


if __name__ == "__main__":
    for p in (W.riemann2d(1024), W.shock_cylinder(), W.mach5_cylinder(), W.sod(200)):
        print(json.dumps(count(p)))
