"""Helpers shared by the tests (no solver arithmetic here)."""
import numpy as np


def normwise_err(a, b):
    """Normwise relative error of a conserved state (or its time derivative) [4, ...]:
    max over quantities of max|a - b| / max|b|, where density and energy are scaled by their
    own maximum and the two momentum components by the maximum of the momentum VECTOR's
    magnitude (a rotation-invariant scale: one component can be round-off-level everywhere,
    e.g. rho*v in gas at rest).  A quantity that is identically zero in b is scaled by the
    largest quantity."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    big = np.abs(b).max()
    mom = np.sqrt(b[1] ** 2 + b[2] ** 2).max()
    scales = [np.abs(b[0]).max(), mom, mom, np.abs(b[3]).max()]
    errs = []
    for c in range(4):
        s = scales[c] if scales[c] > 0 else big
        errs.append(np.abs(a[c] - b[c]).max() / s)
    return max(errs)


def to_dev(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


TOL = 1e-10  # normwise relative error bar on conserved variables
