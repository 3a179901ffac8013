"""Pins for the region-classified unsigned distances and their derivatives."""
import numpy as np
import pytest

from oracle import distance


def _bf_min(point_of, simplex, n=41, levels=12):
    """Brute force: dense grid over the 2-parameter domain, refined around the
    best sample (the squared distance is convex in the parameters)."""
    c = np.array([0.5, 0.5]) if not simplex else np.array([1 / 3, 1 / 3])
    w = 1.0
    best = np.inf
    for _ in range(levels):
        s = np.linspace(c[0] - w, c[0] + w, n)
        t = np.linspace(c[1] - w, c[1] + w, n)
        S, T = np.meshgrid(s, t, indexing="ij")
        S, T = S.ravel(), T.ravel()
        ok = (S >= 0) & (T >= 0) & ((S + T <= 1) if simplex else ((S <= 1) & (T <= 1)))
        S, T = S[ok], T[ok]
        d = point_of(S, T)
        i = np.argmin(d)
        if d[i] < best:
            best = d[i]
        c = np.array([S[i], T[i]])
        w /= 4
    return best


def bf_pt(p, t0, t1, t2):
    f = lambda s, t: np.linalg.norm(p[None] - (t0[None] + s[:, None] * (t1 - t0) + t[:, None] * (t2 - t0)), axis=1)  # noqa
    return _bf_min(f, True)


def bf_ee(a0, a1, b0, b1):
    f = lambda s, t: np.linalg.norm(a0[None] + s[:, None] * (a1 - a0) - b0[None] - t[:, None] * (b1 - b0), axis=1)  # noqa
    return _bf_min(f, False)


def d_of(X4, is_ee):
    reg = distance.classify(X4[None], [is_ee])
    return distance.distances(X4[None], reg)[0], reg[0]


def test_pt_brute_force(rng):
    kinds = set()
    for _ in range(300):
        X4 = rng.normal(size=(4, 3)) * np.array([1.0, 1.0, 0.3])
        X4[0] *= rng.uniform(0.2, 2.0)
        d, reg = d_of(X4, False)
        kinds.add(reg[0])
        assert d == pytest.approx(bf_pt(*X4), rel=1e-6)
    assert kinds == {distance.PP, distance.PE, distance.PT}


def test_ee_brute_force(rng):
    kinds = set()
    for _ in range(300):
        X4 = rng.normal(size=(4, 3))
        d, reg = d_of(X4, True)
        kinds.add(reg[0])
        assert d == pytest.approx(bf_ee(*X4), rel=1e-6)
    assert kinds == {distance.PP, distance.PE, distance.EE}


def test_parallel_edges_fall_back_to_point_edge():
    X4 = np.array([[0, 0, 0], [1, 0, 0], [0.3, 0.002, 0], [1.3, 0.002, 0]], float)
    d, reg = d_of(X4, True)
    assert reg[0] in (distance.PE, distance.PP) and d == pytest.approx(0.002, rel=1e-12)


def test_hand_cases():
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    d, reg = d_of(np.vstack([[0.2, 0.3, 0.005], tri]), False)   # above the face
    assert reg == (distance.PT, (0, 1, 2, 3)) and d == pytest.approx(0.005, rel=1e-14)
    d, reg = d_of(np.vstack([[-0.003, -0.004, 0.0], tri]), False)  # beyond vertex t0
    assert reg == (distance.PP, (0, 1)) and d == pytest.approx(0.005, rel=1e-14)
    d, reg = d_of(np.vstack([[0.5, -0.002, 0.0], tri]), False)   # beside edge t0t1
    assert reg == (distance.PE, (0, 1, 2)) and d == pytest.approx(0.002, rel=1e-14)
    X4 = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0.004], [0, 1, 0.004]], float)  # crossing
    d, reg = d_of(X4, True)
    assert reg[0] == distance.EE and d == pytest.approx(0.004, rel=1e-14)


def test_permutation_symmetry(rng):
    for _ in range(50):
        X4 = rng.normal(size=(4, 3))
        d, _ = d_of(X4, False)
        assert d == pytest.approx(d_of(X4[[0, 2, 3, 1]], False)[0], rel=1e-12)
        assert d == pytest.approx(d_of(X4[[0, 3, 2, 1]], False)[0], rel=1e-12)
        e, _ = d_of(X4, True)
        for perm in ([1, 0, 2, 3], [0, 1, 3, 2], [2, 3, 0, 1]):
            assert e == pytest.approx(d_of(X4[perm], True)[0], rel=1e-10)


def test_continuity_across_regions():
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    ys = np.linspace(-0.01, 0.01, 201)
    ds = [d_of(np.vstack([[0.4, y, 0.003], tri]), False)[0] for y in ys]
    assert np.max(np.abs(np.diff(ds))) < 2 * (ys[1] - ys[0])


def test_derivatives_fd(rng):
    for is_ee in (False, True):
        for _ in range(40):
            X4 = rng.normal(size=(4, 3))
            reg = distance.classify(X4[None], [is_ee])
            d, g, H = distance.distance_derivatives(X4[None], reg)
            h = 1e-6
            f = lambda X: distance.distances(X[None], reg)[0]  # noqa: E731
            for a in range(12):
                dx = np.zeros(12)
                dx[a] = h
                fd = (f(X4 + dx.reshape(4, 3)) - f(X4 - dx.reshape(4, 3))) / (2 * h)
                assert g[0, a] == pytest.approx(fd, rel=1e-6, abs=1e-8)
                gp = distance.distance_derivatives((X4 + dx.reshape(4, 3))[None], reg)[1][0]
                gm = distance.distance_derivatives((X4 - dx.reshape(4, 3))[None], reg)[1][0]
                assert np.allclose(H[0, :, a], (gp - gm) / (2 * h), rtol=1e-5, atol=1e-6)
            assert np.allclose(H[0], H[0].T, atol=1e-10)
            assert d[0] == pytest.approx(f(X4), rel=1e-14)
