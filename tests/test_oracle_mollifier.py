"""Pins for the edge-edge mollifier of the oracle's contact terms.

Reading: the paper uses IPC's clamped log barrier and is silent on parallel
edges; IPC (Li et al. 2020, Sec. 4.3) scales every edge-edge term by
m(c) = (2 - c/eps_x) c/eps_x for c = |u x v|^2 < eps_x = 1e-3 |u_rest|^2 |v_rest|^2
(1 above), because the segment-segment distance is not C^1 where the edges
turn parallel. The pins: the closed form of m, its C^1 join at eps_x, zero
energy and force for exactly parallel edges, finite differences of the
mollified gradient and Hessian, and no change where c >= eps_x."""
import types

import numpy as np
import pytest

from oracle import barrier, contact

DHAT = 1e-3


def _scene(rest):
    return types.SimpleNamespace(X=np.asarray(rest, dtype=np.float64),
                                 edges=np.array([[0, 1], [2, 3]], dtype=np.int32),
                                 tris=np.zeros((0, 3), dtype=np.int32))


def _edges(L1, L2, theta, gap, shift=0.0, tilt=0.0):
    """Edge a along x; edge b at angle theta to it in the xz-plane, gap above in
    y, shifted by `shift` along x and tilted out of plane by `tilt`."""
    a0, a1 = np.array([0.0, 0.0, 0.0]), np.array([L1, 0.0, 0.0])
    c = np.array([0.5 * L1 + shift, gap, 0.0])
    dvec = np.array([np.cos(theta), np.sin(tilt), np.sin(theta)])
    dvec = dvec / np.linalg.norm(dvec)
    return np.stack([a0, a1, c - 0.5 * L2 * dvec, c + 0.5 * L2 * dvec])


def _terms(X4, rest, inA=True, inAp=False, mu=0.0, sigma=3.0):
    sc = _scene(rest)
    e, g, H, _, d = contact.contact_terms(X4, [(1, 0, 1)], sc, np.array([inA]), np.array([inAp]),
                                          np.array([mu]), np.array([0.0]), sigma, DHAT, project=False)
    return e[0], g[0], H[0], d[0]


def test_mollifier_closed_form_and_c1_join():
    L1, L2 = 0.01, 0.012
    rest = _edges(L1, L2, 0.3, 5e-4)
    eps = contact.MOLLIFIER_EPS * L1 ** 2 * L2 ** 2
    for r, want in [(0.0, 0.0), (0.25, 0.4375), (0.5, 0.75), (0.999999, 1.0), (2.0, 1.0)]:
        theta = np.arcsin(np.sqrt(r * eps) / (L1 * L2))
        X4 = _edges(L1, L2, theta, 5e-4)
        m = contact.mollifier(X4[None], np.array([eps]), derivs=False)[0]
        assert m == pytest.approx(want, abs=2e-6)
    # C^1 at c = eps: the one-sided slopes of m in c agree (both zero)
    for side in (-1.0, 1.0):
        r0 = 1.0 + side * 1e-4
        X4a = _edges(L1, L2, np.arcsin(np.sqrt(r0 * eps) / (L1 * L2)), 5e-4)
        X4b = _edges(L1, L2, np.arcsin(np.sqrt((r0 + side * 1e-4) * eps) / (L1 * L2)), 5e-4)
        ma, mb = (contact.mollifier(X[None], np.array([eps]), derivs=False)[0] for X in (X4a, X4b))
        assert abs(mb - ma) / 1e-4 < 1e-3


def test_exactly_parallel_edges_carry_no_energy_or_force():
    rest = _edges(0.01, 0.012, 0.3, 5e-4)
    X4 = _edges(0.01, 0.012, 0.0, 4e-4)
    e, g, H, d = _terms(X4, rest, inAp=True, mu=0.2)
    assert d == pytest.approx(4e-4, rel=1e-12)
    assert e == 0.0
    assert np.abs(g).max() == 0.0


@pytest.mark.parametrize("theta,shift,tilt,inAp", [(2e-3, 0.0, 0.0, False), (5e-4, 0.003, 1e-3, True),
                                                   (1e-3, 0.009, 0.0, False), (3e-3, -0.004, 2e-3, True)])
def test_mollified_edge_edge_terms_match_finite_differences(theta, shift, tilt, inAp):
    """Inside the mollified zone (c < eps_x), with the distance in the interior
    (EE) or an end (PE/PP) region: gradient = FD of the energy, Hessian = FD of
    the gradient."""
    L1, L2 = 0.01, 0.012
    rest = _edges(L1, L2, 0.5, 5e-4)
    X4 = _edges(L1, L2, theta, 4e-4, shift, tilt)
    eps = contact.MOLLIFIER_EPS * L1 ** 2 * L2 ** 2
    m = contact.mollifier(X4[None], np.array([eps]), derivs=False)[0]
    assert 0.0 < m < 1.0
    e, g, H, d = _terms(X4, rest, inAp=inAp, mu=0.15)
    assert d < DHAT
    rng = np.random.default_rng(int(theta * 1e6))
    h = 1e-9
    for k in rng.choice(12, 6, replace=False):
        dx = np.zeros(12)
        dx[k] = h
        ep = _terms(X4 + dx.reshape(4, 3), rest, inAp=inAp, mu=0.15)
        em = _terms(X4 - dx.reshape(4, 3), rest, inAp=inAp, mu=0.15)
        assert g[k] == pytest.approx((ep[0] - em[0]) / (2 * h), rel=1e-5, abs=1e-9 * np.abs(g).max())
        assert H[:, k] == pytest.approx((ep[1] - em[1]) / (2 * h), rel=1e-4, abs=1e-6 * np.abs(H).max())


def test_outside_the_mollified_zone_the_terms_are_unchanged(monkeypatch):
    L1, L2 = 0.01, 0.012
    rest = _edges(L1, L2, 0.5, 5e-4)
    X4 = _edges(L1, L2, 0.2, 4e-4, 0.001)
    on = _terms(X4, rest, inAp=True, mu=0.15)
    monkeypatch.setattr(contact, "MOLLIFY_EE", False)
    off = _terms(X4, rest, inAp=True, mu=0.15)
    for a, b in zip(on, off):
        np.testing.assert_array_equal(a, b)
    # and the unmollified value is the barrier + AL energy of the distance
    d = off[3]
    want = 3.0 * barrier.b(np.array([d]), DHAT)[0] + 0.15 * (DHAT - d) + 3.0 * barrier.b(np.array([d]), DHAT)[0]
    assert off[0] == pytest.approx(want, rel=1e-14)


def test_point_triangle_pairs_are_not_mollified():
    sc = types.SimpleNamespace(X=np.eye(4), edges=np.array([[0, 1], [2, 3]], dtype=np.int32),
                               tris=np.array([[1, 2, 3]], dtype=np.int32))
    eps = contact.ee_eps([(0, 0, 0), (1, 0, 1)], sc)
    assert eps[0] == 0.0 and eps[1] > 0.0
