"""Pins for Algorithm 1's control in the oracle: sigma0 as the minimiser of
the gradient norm (Sec. 3.4), the sigma schedule under both readings of
Alg. 1 line 16, the four branches of the A' rule (lines 3-6) and the dual
update with the slack re-evaluated (lines 12-15, Sec. 3.2.2)."""
import math

import numpy as np
import pytest

from oracle import bal, system
from paper_2407_00046_b300 import scenes

DHAT = 1e-3


def test_sigma0_minimises_the_gradient_norm():
    """Sec. 3.4: sigma0 = argmin_sigma ||grad E + sigma sum grad b||^2 (b over A,
    s = 0, mu = 0). At the returned value (above the floor) the one-dimensional
    function is stationary and not smaller on either side."""
    sc = scenes.two_cubes(n=2)
    sc.X[sc.body == 1, 1] -= 0.01 - 3e-4
    sc.V0[sc.body == 1, 1] = -3.0              # the upper cube moves onto the lower one
    m = system.make_model(sc)
    y = system.inertia_target(m, sc.X, sc.V0)
    keys, _ = bal.active_pairs(m, sc.X)
    assert len(keys) > 0
    s0 = bal.initial_sigma(m, sc.X, y, keys)
    assert s0 > bal.sigma_floor(m)            # the formula, not the floor
    n = len(keys)
    ps = system.PairSet(keys, np.ones(n, bool), np.zeros(n, bool), np.zeros(n), np.zeros(n))
    _, gE, gb = system.gradient(m, sc.X, y, ps, 1.0, parts=True)

    def f(s):
        r = gE + s * gb
        return float(np.sum(r * r))

    h = 1e-6 * s0
    slope = (f(s0 + h) - f(s0 - h)) / (2 * h)
    curv = (f(s0 + h) - 2 * f(s0) + f(s0 - h)) / h ** 2
    assert abs(slope) <= 1e-6 * curv * s0
    assert f(s0) <= f(0.9 * s0) and f(s0) <= f(1.1 * s0)


def test_sigma0_falls_back_to_the_floor_without_contact():
    sc = scenes.two_cubes(n=2)
    m = system.make_model(sc)
    y = system.inertia_target(m, sc.X, sc.V0)
    assert bal.initial_sigma(m, sc.X, y, []) == bal.sigma_floor(m)


def test_sigma_schedule_printed_rule_and_capped_reading():
    lit = bal.Params(sigma_literal_max=True)
    cap = bal.Params(sigma_literal_max=False)
    s0, close, far = 2.0, 0.5e-2 * DHAT, 2e-2 * DHAT
    # printed rule: jump to 100 sigma0, then grow by 1.2 per iteration without bound
    s = s0
    seq = []
    for _ in range(4):
        s = bal.sigma_update(s, s0, close, lit, DHAT)
        seq.append(s)
    assert seq == pytest.approx([200.0, 240.0, 288.0, 345.6], rel=1e-15)
    # capped reading: grow by 1.2 up to 100 sigma0
    s, k = s0, 0
    while s < 100 * s0 and k < 100:
        s_new = bal.sigma_update(s, s0, close, cap, DHAT)
        assert s_new == pytest.approx(min(1.2 * s, 200.0), rel=1e-15)
        s, k = s_new, k + 1
    assert s == 200.0 and k == math.ceil(math.log(100) / math.log(1.2))
    assert bal.sigma_update(s, s0, close, cap, DHAT) == 200.0
    # no change while every distance is above 1e-2 dhat (and for the empty set)
    for prm in (lit, cap):
        assert bal.sigma_update(7.0, s0, far, prm, DHAT) == 7.0
        assert bal.sigma_update(7.0, s0, math.inf, prm, DHAT) == 7.0


def test_augmentation_set_rule_branches():
    prm = bal.Params()
    thr = 1e-2 * DHAT
    A = [(0, 1, 2), (0, 3, 4), (1, 5, 6), (1, 7, 8)]
    d = np.array([0.5 * thr, 2 * thr, 0.2 * thr, 5 * thr])
    old = {(0, 1, 2): 0.3, (1, 9, 10): 0.7}
    # 1. min d > 1e-2 dhat: A' emptied
    assert bal.augmentation_set(old, A, 2 * d + thr, 1.01 * thr, 0.0, prm, DHAT) == {}
    # 2. min d fell below the previous iterate's: rebuilt from the close pairs,
    #    mu kept for pairs that stay, new pairs start at 0, dropped pairs leave
    new = bal.augmentation_set(old, A, d, d.min(), 0.5 * thr, prm, DHAT)
    assert new == {(0, 1, 2): 0.3, (1, 5, 6): 0.0}
    # 3. A' empty: rebuilt even though min d did not fall
    assert bal.augmentation_set({}, A, d, d.min(), 0.1 * thr, prm, DHAT) == {(0, 1, 2): 0.0, (1, 5, 6): 0.0}
    # 4. min d did not fall and A' is non-empty: kept as it is
    assert bal.augmentation_set(old, A, d, d.min(), d.min(), prm, DHAT) == old
    assert bal.augmentation_set(old, A, d, d.min(), 0.1 * thr, prm, DHAT) == old


def test_dual_update_with_the_slack_re_evaluated():
    """One pair, sigma = 3, mu = 0.2: at d = dhat / e the slack is 0 and
    b(d, dhat) = (dhat - d)^2 (log(d / dhat) = -1), so mu grows by
    3 (dhat (1 - 1/e))^2. A pair beyond dhat, or beyond dhat + mu / sigma (slack
    > 0, so the barrier is evaluated at its own distance), keeps its mu."""
    sigma, mu = 3.0, 0.2
    d = DHAT / math.e
    out = bal.dual_update({(0, 1, 2): mu}, [d], sigma, DHAT)
    assert out[(0, 1, 2)] == pytest.approx(mu + sigma * (DHAT * (1 - 1 / math.e)) ** 2, rel=1e-13)
    for dd in (1.5 * DHAT, DHAT + mu / sigma + 1e-4):
        assert bal.dual_update({(0, 1, 2): mu}, [dd], sigma, DHAT) == {(0, 1, 2): mu}
    # mu = 0 and d < dhat: mu becomes sigma b, and it never decreases
    # (distances in the sorted order of the keys)
    out = bal.dual_update({(1, 4, 5): 0.0, (0, 1, 2): mu}, [0.9 * DHAT, DHAT / math.e], sigma, DHAT)
    assert out[(1, 4, 5)] == pytest.approx(sigma * (DHAT * (1 - 1 / math.e)) ** 2, rel=1e-13)
    assert out[(0, 1, 2)] >= mu
