"""Pins for the time step (Sec. 3.1 / Algorithm 1): closed-form free flight,
linear momentum conservation through contact, and the method's invariants."""
import numpy as np
import pytest

from oracle import bal, contact, elastic, system
from paper_2407_00046_b300 import scenes


def test_free_flight_is_exact():
    X, T = scenes.lattice_box(3, 3, 3, (0.1, 0.1, 0.1))
    sc = scenes.merge_bodies("free", [dict(X=X, tets=T, E=1e5, V0=np.array([0.1, 0.2, -0.3]))])
    m = system.make_model(sc)
    x, v, info = bal.time_step(m, sc.X, sc.V0, bal.Params(newton_tol=1e-12))
    y = system.inertia_target(m, sc.X, sc.V0)
    assert info["converged"]
    assert np.abs(x - y).max() < 1e-13
    assert np.allclose(v, sc.V0 + sc.h * sc.gravity, atol=1e-11)


def _approaching_cubes():
    X0, T0 = scenes.lattice_box(2, 2, 2, (0.05, 0.05, 0.05))
    X1, T1 = scenes.lattice_box(2, 2, 2, (0.05, 0.05, 0.05))
    X1 = X1 + np.array([0.0512, 0.011, 0.007])
    sc = scenes.merge_bodies("approach", [
        dict(X=X0, tets=T0, E=1e5, V0=np.array([0.2, 0.0, 0.0])),
        dict(X=X1, tets=T1, E=3e5, V0=np.array([-0.3, 0.0, 0.05]))])
    sc.gravity = np.zeros(3)
    return sc


def test_momentum_conserved_through_contact():
    sc = _approaching_cubes()
    m = system.make_model(sc)
    x, v = sc.X.copy(), sc.V0.copy()
    p0 = (m.mass[:, None] * v).sum(axis=0)
    saw_contact = False
    for _ in range(3):
        x, v, info = bal.time_step(m, x, v, bal.Params(newton_tol=1e-10, newton_max=300))
        saw_contact |= any(r["nA"] > 0 for r in info["log"])
        p = (m.mass[:, None] * v).sum(axis=0)
        assert np.abs(p - p0).max() < 1e-8 * np.abs(p0).max()
    assert saw_contact


def test_invariants_after_each_step():
    sc = scenes.two_cubes(n=2)
    m = system.make_model(sc)
    x, v = sc.X.copy(), sc.V0.copy()
    for _ in range(3):
        xo = x
        x, v, info = bal.time_step(m, x, v, bal.Params(newton_tol=1e-6))
        F = elastic.deformation_gradient(x, sc.tets, m.Dm_inv)
        assert np.linalg.det(F).min() > 0                                  # inversion-free
        cand = contact.candidate_pairs(x, sc, 2 * sc.dhat)
        d, _, _ = contact.pair_distances(x, cand, sc)
        assert d.size == 0 or d.min() > 0                                  # intersection-free
        assert np.all(x[sc.pinned == 1] == xo[sc.pinned == 1])             # Dirichlet
        for r in info["log"]:
            assert r.get("alpha", 1.0) > 0


def _pt_scene():
    # one vertex (tiny tet) above a large triangle face (flat slab)
    Xs, Ts = scenes.lattice_box(1, 1, 1, (0.2, 0.05, 0.2))
    Xp, Tp = scenes.lattice_box(1, 1, 1, (0.01, 0.01, 0.01))
    Xp = Xp + np.array([0.07, 0.05 + 0.004, 0.06])
    return scenes.merge_bodies("pt", [dict(X=Xs, tets=Ts, E=1e5), dict(X=Xp, tets=Tp, E=1e5)])


def test_step_bound_head_on_closed_form():
    sc = _pt_scene()
    m = system.make_model(sc)
    p = np.zeros_like(sc.X)
    p[sc.body == 1] = [0.0, -0.02, 0.0]        # closes 2 cm per unit step at a 4 mm gap
    cand = contact.candidate_pairs(sc.X, sc, 0.05)
    alpha = bal.step_bound(m, sc.X, p, cand, bal.Params())
    assert alpha == pytest.approx(0.9 * 0.004 / 0.02, rel=1e-9)


def test_step_bound_sliding_is_not_limited():
    sc = _pt_scene()
    m = system.make_model(sc)
    p = np.zeros_like(sc.X)
    p[sc.body == 1] = [0.03, 0.0, 0.02]          # tangential motion over the face
    cand = contact.candidate_pairs(sc.X, sc, 0.05)
    assert bal.step_bound(m, sc.X, p, cand, bal.Params()) == 1.0
    p[sc.body == 1] = [0.03, -0.002, 0.02]       # mostly sliding, slowly closing: not limited either
    assert bal.step_bound(m, sc.X, p, cand, bal.Params()) == 1.0
