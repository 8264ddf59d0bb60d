"""Host logic of the inverse driver (Sec. 3 gamma recovery, Sec. 2.4 multi-step loss): the
learning-rate schedule, the loss and the gamma dependence of the initial state, on CPU."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2601_04400_gb300 import inverse as I


def test_warm_cosine_schedule():
    f = lambda k: I.warm_cosine(k, 200, 1200, 1e-6, 1e-8)
    assert f(0) == 1e-6 and f(199) == 1e-6 and f(200) == 1e-6
    assert f(1200) == pytest.approx(1e-8, rel=1e-15) and f(5000) == pytest.approx(1e-8, rel=1e-15)
    assert f(700) == pytest.approx(0.5 * (1e-6 + 1e-8), rel=1e-14)   # half way: the mean
    vals = [f(k) for k in range(200, 1201)]
    assert all(a >= b for a, b in zip(vals, vals[1:]))               # monotone decay
    # cosine shape: lr(warm + t T) = lr_end + (lr_start - lr_end)(1 + cos(pi t)) / 2
    assert f(450) == pytest.approx(1e-8 + (1e-6 - 1e-8) * (1 + math.cos(math.pi / 4)) / 2, rel=1e-14)


def test_multistep_loss_is_the_mean_of_the_step_losses():
    rng = np.random.default_rng(0)
    S = rng.standard_normal((5, 4, 3, 7))
    T = rng.standard_normal((5, 4, 3, 7))
    mask = rng.random((3, 7)) < 0.5
    got = float(I.multistep_loss(torch.tensor(S), torch.tensor(T), torch.tensor(mask)))
    ref = np.mean([sum(((S[s, c] - T[s, c])[mask] ** 2).sum() for c in range(4)) for s in range(5)])
    assert got == pytest.approx(ref, rel=1e-14)
    got_all = float(I.multistep_loss(torch.tensor(S), torch.tensor(T)))
    assert got_all == pytest.approx(((S - T) ** 2).sum() / 5, rel=1e-14)


