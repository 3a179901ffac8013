"""Pins for the IPC clamped log barrier (Sec. 3.3, Eq. IPC-barrier)."""
import math

import numpy as np
import pytest

from oracle import barrier

DH = 1e-3


def test_c2_clamp_at_offset():
    for c in (DH, 2.5e-3):
        d = np.array([c, c * (1 + 1e-12), 2 * c])
        assert np.all(barrier.b(d, c) == 0) and np.all(barrier.db(d, c) == 0)
        assert np.all(barrier.d2b(d, c) == 0)
        # approaching from below: b ~ e^3/c, b' ~ 3 e^2/(2c)... all vanish (C^2)
        e = c * 1e-6
        assert abs(barrier.b(np.array([c - e]), c)[0]) < 2 * e ** 3 / c
        assert abs(barrier.db(np.array([c - e]), c)[0]) < 4 * e ** 2 / c
        assert abs(barrier.d2b(np.array([c - e]), c)[0]) < 8 * e / c


def test_hand_values():
    # b(c/2, c) = -(c/2)^2 ln(1/2) = c^2 ln2 / 4
    assert barrier.b(np.array([DH / 2]), DH)[0] == pytest.approx(DH ** 2 * math.log(2) / 4, rel=1e-15)
    # b''(c/2, c) = 2 ln 2 + 5 (dimensionless)
    assert barrier.d2b(np.array([DH / 2]), DH)[0] == pytest.approx(2 * math.log(2) + 5, rel=1e-14)
    # b'(c/2, c) = c ln(1/2) ... = -2(-c/2) ln(1/2) - (c/2)^2/(c/2) = -c ln 2 - c/2
    assert barrier.db(np.array([DH / 2]), DH)[0] == pytest.approx(-DH * math.log(2) - DH / 2, rel=1e-14)


def test_convex_repulsive_on_support():
    d = np.geomspace(1e-9, DH * (1 - 1e-9), 400)
    assert np.all(barrier.d2b(d, DH) > 0)
    assert np.all(barrier.db(d, DH) < 0)
    assert np.all(barrier.b(d, DH) > 0)
    assert barrier.b(np.array([0.0]), DH)[0] == np.inf


@pytest.mark.parametrize("scale", [1e-6, 1e-5, 1e-4, 5e-4, 9.9e-4])
def test_fd(scale):
    for c in (DH, 1.7e-3):
        d = scale * c / 1e-3
        h = d * 1e-6
        fd1 = (barrier.b(np.array([d + h]), c)[0] - barrier.b(np.array([d - h]), c)[0]) / (2 * h)
        fd2 = (barrier.db(np.array([d + h]), c)[0] - barrier.db(np.array([d - h]), c)[0]) / (2 * h)
        assert barrier.db(np.array([d]), c)[0] == pytest.approx(fd1, rel=1e-7)
        assert barrier.d2b(np.array([d]), c)[0] == pytest.approx(fd2, rel=1e-7)
