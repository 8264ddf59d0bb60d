"""Parity at the two full-size benchmark configurations over their FULL step counts, against
reference runs of the oracle stored in tests/golden (written by
tests/golden/make_fullrun_goldens.py, which calls only the oracle: CPU hours, so not at test
time):

* the viscous Mach-2 shock over the immersed cylinder, 2048 x 1024, 2000 CFL steps;
* the four-quadrant Riemann problem, 1024 x 1024, CFL steps to t = 0.8 (the last one clipped).

The IEEE-order arithmetic mode (js_set_arith JS_ARITH_IEEE) must reproduce both runs BIT FOR
BIT: SHA-256 digests of the state (float64 bytes of [4][ny][nx]) and of the step sizes equal
the oracle's at every checkpoint, to the end.  The default fast kernel must equal the oracle's
sampled cells within the parity bar (1e-10 of each quantity's maximum) after the cylinder's 2000
steps, and after 1000 steps of the four-quadrant problem (beyond that, its shear layers amplify
differences of one unit in the last place exponentially: any two FP64 implementations that
round differently part, which the opt-in 1-ulp control runs of test_gpu_fullrun.py show; the
IEEE mode, which rounds exactly as the oracle, does not)."""
import hashlib
import os

import numpy as np
import pytest

import oracle as O
from paper_2601_04400_gb300 import workloads as W
from jsutil import TOL

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04400_gb300 import binding
    binding.lib()
    return binding


def load_golden(name):
    """{'steps': n, 'checkpoints': {k: dict(t, state, dts, scale)}, 'samples': {k: (j, i, values)}}"""
    cps, samples, steps = {}, {}, None
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            w = line.split()
            if not w or w[0].startswith("#"):
                continue
            if w[0] == "checkpoint":
                k = int(w[1])
                cps[k] = dict(t=float(w[3]), state=w[5], dts=w[7], scale=[float(v) for v in w[9:12]])
            elif w[0] == "sample":
                k = int(w[1])
                samples.setdefault(k, []).append((int(w[2]), int(w[3]), [float(v) for v in w[4:8]]))
            elif w[0] == "steps":
                steps = int(w[1])
    out = {"steps": steps, "checkpoints": cps, "samples": {}}
    for k, rows in samples.items():
        out["samples"][k] = (np.array([r[0] for r in rows]), np.array([r[1] for r in rows]),
                             np.array([r[2] for r in rows]).T)
    return out


def sha256(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<f8").tobytes()).hexdigest()


def sampled_err(U, g, k):
    """Normwise error on the sampled cells: per quantity max |a - b| / (the oracle's maximum over
    the whole grid; the momentum components share the momentum vector's)."""
    j, i, ref = g["samples"][k]
    got = U[:, j, i]
    sc = g["checkpoints"][k]["scale"]
    scale = [sc[0], sc[1], sc[1], sc[2]]
    return max(np.abs(got[c] - ref[c]).max() / scale[c] for c in range(4))


def run(B, prob, g, ieee, stop_at=None):
    """CFL steps on the device (js_step_cfl) in chunks up to each checkpoint; returns
    {k: (state, dts so far, t)}."""
    import torch
    s = B.Solver.from_problem(prob)
    if ieee:
        s.set_arith("ieee")
    U = torch.tensor(O.prim_to_cons(prob, prob.W0), device="cuda")
    t = torch.zeros((), dtype=torch.float64, device="cuda")
    t_end = prob.t_end if prob.t_end is not None else 0.0
    dts, done, out = [], 0, {}
    for k in sorted(g["checkpoints"]):
        if stop_at is not None and k > stop_at:
            break
        n = k - done
        log = torch.zeros(n, dtype=torch.float64, device="cuda")
        s.step_cfl(U, prob.cfl, n, t=t, t_end=t_end, dt_log=log)
        lg = log.cpu().numpy()
        assert (lg > 0).all(), "a step did nothing before the checkpoint"
        dts.extend(lg.tolist())
        done = k
        out[k] = (U.cpu().numpy(), np.array(dts), float(t))
    assert s.status() == 0
    s.close()
    return out


CASES = [("shock_cylinder", lambda: W.shock_cylinder(), "fullrun_shock_cylinder_2048x1024.txt", None),
         ("riemann2d", lambda: W.riemann2d(1024), "fullrun_riemann2d_1024.txt", 1000)]


@pytest.mark.parametrize("name,make,golden,fast_until", CASES, ids=[c[0] for c in CASES])
def test_ieee_mode_reproduces_the_oracle_run_bit_for_bit(B, name, make, golden, fast_until):
    g = load_golden(golden)
    prob = make()
    res = run(B, prob, g, ieee=True)
    assert max(res) == g["steps"]
    for k, (U, dts, t) in sorted(res.items()):
        cp = g["checkpoints"][k]
        assert sha256(dts) == cp["dts"], "step sizes differ by checkpoint %d" % k
        assert t == cp["t"]
        assert sha256(U) == cp["state"], "state differs at checkpoint %d (sampled error %.3e)" % (
            k, sampled_err(U, g, k))


@pytest.mark.parametrize("name,make,golden,fast_until", CASES, ids=[c[0] for c in CASES])
def test_fast_kernel_matches_the_oracle_run(B, name, make, golden, fast_until):
    g = load_golden(golden)
    prob = make()
    res = run(B, prob, g, ieee=False, stop_at=fast_until)
    for k, (U, dts, t) in sorted(res.items()):
        cp = g["checkpoints"][k]
        assert abs(t - cp["t"]) <= 1e-11 * cp["t"]
        err = sampled_err(U, g, k)
        print("%s checkpoint %d: sampled normwise error %.3e" % (name, k, err))
        assert err < TOL, (k, err)
