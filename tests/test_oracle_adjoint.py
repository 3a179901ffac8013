"""Pins for the FP64 oracle adjoint: free-flight closed form and central
finite differences through contact."""
import numpy as np
import pytest

from oracle import adjoint, bal, system
from paper_2407_00046_b300 import scenes


def _loss(model, xT, body, target):
    m = model.mass[body]
    c = (m[:, None] * xT[body]).sum(0) / m.sum()
    r = c - target
    g = np.zeros_like(xT)
    g[body] = 2.0 * r[None, :] * (m[:, None] / m.sum())
    return float(r @ r), g


def test_free_flight_velocity_gradient_closed_form():
    X, T = scenes.lattice_box(2, 2, 2, (0.05, 0.05, 0.05))
    sc = scenes.merge_bodies("free", [dict(X=X, tets=T, E=1e5, V0=np.array([0.1, 0.0, -0.2]))])
    model = system.make_model(sc)
    steps = 3
    prm = bal.Params(newton_tol=1e-12)
    xT, vT, ck = adjoint.forward(model, sc.X, sc.V0, steps, prm)
    body = np.arange(sc.n_verts)
    target = np.array([0.3, -0.1, 0.2])
    J, gx = _loss(model, xT, body, target)
    dx0, dv0, dE = adjoint.backward(model, ck, gx, np.zeros_like(gx))
    c = (model.mass[:, None] * xT).sum(0) / model.mass.sum()
    expect = 2 * steps * sc.h * (model.mass[:, None] / model.mass.sum()) * (c - target)[None, :]
    assert np.allclose(dv0, expect, rtol=1e-9, atol=1e-14)
    assert np.abs(dE).max() < 1e-12 * max(1.0, np.abs(dv0).max())


def _contact_case():
    sc = scenes.cube_on_slab(n_cube=2, slab_cells=(3, 1, 3), slab_size=(0.2, 0.04, 0.2), gap=0.004,
                             E_cube=2e4, E_slab=1e5)
    return sc, system.make_model(sc)


def test_adjoint_matches_central_fd_through_contact():
    sc, model = _contact_case()
    prm = bal.Params(newton_tol=1e-12, newton_max=400)
    steps = 2
    body = np.flatnonzero(sc.body == 0)
    target = sc.info["target"]
    xT, _, ck = adjoint.forward(model, sc.X, sc.V0, steps, prm)
    _, _, info = bal.time_step(model, ck[-1][0], (ck[-1][0] - ck[-2][0]) / sc.h, prm)
    assert max(r["nA"] for r in info["log"]) > 0          # the cube is in contact
    J, gx = _loss(model, xT, body, target)
    _, dv0, dE = adjoint.backward(model, ck, gx, np.zeros_like(gx))
    frozen = [(c[3], c[4]) for c in ck]     # perturbed runs keep each step's AL state
    rng = np.random.default_rng(0)
    # directional derivative in E: J(E (1 + eps w))
    w = rng.choice([-1.0, 1.0], size=sc.n_tets)
    E0 = sc.E.copy()
    eps = 1e-4
    vals = []
    for sgn in (1, -1):
        sc.E[:] = E0 * (1 + sgn * eps * w)
        m2 = system.make_model(sc)
        x2, _, _ = adjoint.forward(m2, sc.X, sc.V0, steps, prm, frozen)
        vals.append(_loss(m2, x2, body, target)[0])
    sc.E[:] = E0
    fd = (vals[0] - vals[1]) / (2 * eps)
    assert np.sum(dE * E0 * w) == pytest.approx(fd, rel=1e-4)
    # directional derivative in v0 over the cube vertices
    u = np.zeros_like(sc.V0)
    u[body] = rng.normal(size=(len(body), 3))
    vals = []
    for sgn in (1, -1):
        x2, _, _ = adjoint.forward(model, sc.X, sc.V0 + sgn * 1e-6 * u, steps, prm, frozen)
        vals.append(_loss(model, x2, body, target)[0])
    fd = (vals[0] - vals[1]) / 2e-6
    assert np.sum(dv0 * u) == pytest.approx(fd, rel=1e-5)
