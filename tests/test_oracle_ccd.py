"""Pins of the oracle's cubic CCD (Sec. 5.3): closed-form crossings, the root
finder against numpy's companion-matrix roots, and a dense time scan of random
moving stencils."""
import numpy as np
import pytest

from oracle import ccd, distance

DHAT = 1e-3


def _pt(p, t0, t1, t2):
    return np.array([p, t0, t1, t2], dtype=float)


TRI = ([0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0])


def test_vertex_falling_through_triangle_hits_at_half_step():
    X = _pt([0.2, 0.1, 0.2], *TRI)
    P = np.zeros((4, 3))
    P[0] = [0.0, -0.2, 0.0]                      # crosses y = 0 at t = 0.5
    toi = ccd.pair_toi(X, P, False, DHAT)
    assert 0.45 - 1e-12 <= toi <= 0.5
    f = ccd.cubic_coefficients(X[None], P[None], False)[0]
    assert np.sign(ccd._poly(f, toi)) == np.sign(ccd._poly(f, 0.0))


def test_step_bound_applies_the_margin_to_activated_pairs_only():
    X = _pt([0.2, 0.1, 0.2], *TRI)
    P = np.zeros((4, 3))
    P[0] = [0.0, -0.2, 0.0]
    raw = ccd.pair_toi(X, P, False, DHAT)
    assert ccd.pair_toi(X, P, False, DHAT, eta=0.9) == pytest.approx(0.9 * raw, rel=1e-15)
    Q = P.copy()
    Q[0] = [0.3, 0.0, 0.0]                       # parallel motion: no activation, no margin
    assert ccd.pair_toi(X, Q, False, DHAT, eta=0.9) == 1.0


def test_vertex_passing_beside_triangle_does_not_activate():
    X = _pt([2.0, 0.1, 2.0], *TRI)               # crosses the plane far outside the triangle
    P = np.zeros((4, 3))
    P[0] = [0.0, -0.2, 0.0]
    assert ccd.pair_toi(X, P, False, DHAT) == 1.0


def test_vertex_passing_within_dhat_of_an_edge_activates():
    X = _pt([0.5 + 0.5 * DHAT, 0.1, -0.5 * DHAT], *TRI)   # just outside edge t0 t1, within dhat
    P = np.zeros((4, 3))
    P[0] = [0.0, -0.2, 0.0]
    toi = ccd.pair_toi(X, P, False, DHAT)
    assert 0.45 - 1e-12 <= toi <= 0.5
    X[0, 2] = -2.0 * DHAT                        # now beyond dhat: no activation
    assert ccd.pair_toi(X, P, False, DHAT) == 1.0


def test_crossing_edges_closed_form():
    # edge a along x at y = 0; edge b along z at y = 0.3 moving down at 0.4 per step
    X = np.array([[-1.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.3, -1.0], [0.0, 0.3, 1.0]])
    P = np.zeros((4, 3))
    P[2:, 1] = -0.4                              # crossing at t = 0.75
    toi = ccd.pair_toi(X, P, True, DHAT)
    assert 0.9 * 0.75 - 1e-12 <= toi <= 0.75


def test_motion_parallel_to_the_plane_never_crosses():
    X = _pt([0.2, 0.1, 0.2], *TRI)
    P = np.zeros((4, 3))
    P[0] = [0.3, 0.0, -0.1]
    assert ccd.pair_toi(X, P, False, DHAT) == 1.0


def test_identically_coplanar_stencil_does_not_bound_the_step():
    X = _pt([2.0, 0.0, 2.0], *TRI)               # in the triangle's plane, sliding in it
    P = np.zeros((4, 3))
    P[0] = [-0.5, 0.0, -0.5]
    assert ccd.pair_toi(X, P, False, DHAT) == 1.0


def test_roots_match_numpy_companion_roots():
    rng = np.random.default_rng(0)
    checked = 0
    for _ in range(2000):
        r = np.sort(rng.uniform(-0.5, 1.5, size=3))
        a = rng.choice([-1.0, 1.0]) * 10 ** rng.uniform(-3, 3)
        c = a * np.array([-r[0] * r[1] * r[2], r[0] * r[1] + r[1] * r[2] + r[0] * r[2],
                          -(r[0] + r[1] + r[2]), 1.0])
        got = ccd.coplanar_times(c)
        ref = np.roots(c[::-1])
        ref = np.sort(ref[np.abs(ref.imag) < 1e-9].real)
        ref = ref[(ref >= -ccd.EPS) & (ref <= 1 + ccd.EPS)]
        if np.min(np.diff(r)) < 1e-6:
            continue
        assert len(got) == len(ref), (r, got, ref)
        assert np.allclose(got, ref, rtol=0, atol=1e-9), (got, ref)
        checked += 1
    assert checked > 1500


@pytest.mark.parametrize("is_ee", [False, True])
def test_toi_against_a_dense_time_scan(is_ee):
    """The first sign change of f whose stencil distance is below dhat, found by
    scanning t on a fine grid, brackets the conservative TOI from above; the
    TOI keeps the pre-crossing side."""
    rng = np.random.default_rng(3 if is_ee else 4)
    ts = np.linspace(0.0, 1.0, 20001)
    hits = 0
    for _ in range(300):
        X = rng.normal(size=(4, 3)) * 0.05
        P = rng.normal(size=(4, 3)) * 0.08
        c = ccd.cubic_coefficients(X[None], P[None], is_ee)[0]
        f = ccd._poly(c, ts)
        sc = np.flatnonzero(np.sign(f[1:]) != np.sign(f[:-1]))
        t_first, first_is_act = None, False
        for n, k in enumerate(sc):
            tc = 0.5 * (ts[k] + ts[k + 1])
            Xt = (X + tc * P)[None]
            d = distance.distances(Xt, distance.classify(Xt, np.array([is_ee])))[0]
            if d < 0.5 * DHAT:          # clearly activated (the scan has finite resolution)
                t_first, first_is_act = ts[k + 1], n == 0
                break
            if d > 2 * DHAT:            # clearly not
                continue
            t_first = -1.0              # ambiguous within the grid resolution: skip
            break
        toi = ccd.pair_toi(X, P, is_ee, DHAT)
        assert 0.0 <= toi <= 1.0
        if t_first is None:
            assert toi == 1.0
            continue
        if t_first < 0:
            continue
        hits += 1
        assert toi <= t_first + 1e-12
        assert ccd._poly(c, toi) != 0.0
        if first_is_act:                # before the first crossing: the side of t = 0
            assert np.sign(ccd._poly(c, toi)) == np.sign(ccd._poly(c, 0.0))
    assert hits > 5


def test_ccd_and_ca_line_searches_reach_the_same_minimiser():
    """With the AL state held fixed (sigma, A' = {}), the step bound changes
    only the Newton path, not the minimiser of L_sigma: with a tight Newton
    tolerance both line searches land on the same positions, and every contact
    distance stays positive."""
    from oracle import bal, system
    from paper_2407_00046_b300 import scenes
    sc = scenes.two_cubes(n=2)
    sc.X[sc.body == 1, 1] -= 0.01 - 5e-4
    m = system.make_model(sc)
    out = {}
    for mode in ("ca", "ccd"):
        x, v, info = bal.time_step(m, sc.X.copy(), sc.V0.copy(),
                                   bal.Params(newton_tol=1e-11, step_mode=mode), frozen=(5.0, {}))
        assert info["converged"]
        keys, d = bal.active_pairs(m, x)
        assert len(d) > 0 and d.min() > 0.0
        out[mode] = x
    assert np.abs(out["ca"] - out["ccd"]).max() < 1e-9
