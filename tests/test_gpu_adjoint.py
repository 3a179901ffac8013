"""GPU adjoint of the time step (not in the paper): closed form, oracle parity
on the same checkpoints, and central finite differences with the AL state of
each step held fixed (the map the adjoint differentiates)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import adjoint as oadj  # noqa: E402
from oracle import bal as obal  # noqa: E402
from oracle import system  # noqa: E402
from paper_2407_00046_b300 import bal, scenes  # noqa: E402
from paper_2407_00046_b300.autograd import simulate  # noqa: E402

DEV = "cuda"


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def centroid_loss(xT, mass, body, target):
    m = mass[body]
    c = (m[:, None] * xT.view(-1, 3)[body]).sum(0) / m.sum()
    return ((c - target) ** 2).sum()


def _params(**kw):
    return bal.default_params(newton_tol=1e-12, newton_max_iter=400, pcg_tol=1e-13,
                              pcg_max_iter=50000, **kw)


def test_free_flight_velocity_gradient_closed_form():
    X, Tt = scenes.lattice_box(2, 2, 2, (0.05, 0.05, 0.05))
    sc = scenes.merge_bodies("free", [dict(X=X, tets=Tt, E=1e5, V0=np.array([0.1, 0.0, -0.2]))])
    S = bal.Scene(sc, _params())
    mass = torch.tensor(S.mass(), device=DEV)
    body = torch.arange(sc.n_verts, device=DEV)
    target = T([0.3, -0.1, 0.2])
    E = T(sc.E).requires_grad_(True)
    v0 = T(sc.V0).view(-1).requires_grad_(True)
    x0 = T(sc.X).view(-1)
    steps = 3
    xT, vT = simulate(S, x0, v0, E, steps)
    J = centroid_loss(xT, mass, body, target)
    J.backward()
    c = (mass[:, None] * xT.view(-1, 3)).sum(0) / mass.sum()
    expect = 2 * steps * sc.h * (mass[:, None] / mass.sum()) * (c - target)[None, :]
    assert torch.allclose(v0.grad.view(-1, 3), expect, rtol=1e-9, atol=1e-14)
    assert float(E.grad.abs().max()) < 1e-12 * max(1.0, float(v0.grad.abs().max()))


def _contact_case():
    sc = scenes.cube_on_slab(n_cube=2, slab_cells=(3, 1, 3), slab_size=(0.2, 0.04, 0.2), gap=0.004,
                             E_cube=2e4, E_slab=1e5)
    return sc


def _rollout(S, sc, steps, frozen=None, E=None, V0=None):
    if E is not None:
        S.set_materials(E)
    x, v = T(sc.X).view(-1), T(sc.V0 if V0 is None else V0).view(-1)
    ck = []
    for k in range(steps):
        xt, vt = x.clone(), v.clone()
        if frozen is not None:
            S.set_params(freeze_al=1)
            S.set_al_state(frozen[k]["sigma"], frozen[k]["sigma0"], frozen[k]["ap_keys"], frozen[k]["ap_mu"])
        info = S.time_step(x, v)
        assert info["converged"] == 1
        ck.append((xt, vt, x.clone(), S.get_al_state()))
    S.set_params(freeze_al=0)
    return x, ck


def test_adjoint_matches_oracle_on_the_same_checkpoints():
    sc = _contact_case()
    S = bal.Scene(sc, _params())
    steps = 2
    xT, ck = _rollout(S, sc, steps)
    m = system.make_model(sc)
    body = np.flatnonzero(sc.body == 0)
    target = sc.info["target"]
    mass = torch.tensor(S.mass(), device=DEV)
    xg = xT.clone().requires_grad_(True)
    J = centroid_loss(xg, mass, torch.tensor(body, device=DEV), T(target))
    J.backward()
    gx = xg.grad.clone()
    gv = torch.zeros_like(gx)
    dE = torch.zeros(sc.n_tets, dtype=torch.float64, device=DEV)
    gxo, gvo = gx.cpu().numpy().reshape(-1, 3), np.zeros((sc.n_verts, 3))
    dEo = np.zeros(sc.n_tets)
    saw_contact = False
    for xt, vt, xn, al in reversed(ck):
        gx, gv, info = S.adjoint_step(xt, vt, xn, al, gx, gv, dE)
        Ap = {bal.unpack_key(k): mu for k, mu in zip(al["ap_keys"], al["ap_mu"])}
        keys, _ = obal.active_pairs(m, xn.cpu().numpy().reshape(-1, 3))
        saw_contact |= len(keys) > 0
        gxo, gvo, de = oadj.step_adjoint(m, xt.cpu().numpy().reshape(-1, 3), vt.cpu().numpy().reshape(-1, 3),
                                         xn.cpu().numpy().reshape(-1, 3), al["sigma"], Ap, gxo, gvo)
        dEo += de
    assert saw_contact
    for a, b in ((gx.cpu().numpy().reshape(-1, 3), gxo), (gv.cpu().numpy().reshape(-1, 3), gvo),
                 (dE.cpu().numpy(), dEo)):
        assert np.abs(a - b).max() <= 1e-7 * np.abs(b).max() + 1e-300


def test_adjoint_matches_central_fd_with_frozen_al_state():
    sc = _contact_case()
    S = bal.Scene(sc, _params())
    steps = 2
    body = torch.tensor(np.flatnonzero(sc.body == 0), device=DEV)
    target = T(sc.info["target"])
    mass = torch.tensor(S.mass(), device=DEV)
    E = T(sc.E).requires_grad_(True)
    v0 = T(sc.V0).view(-1).requires_grad_(True)
    xT, vT = simulate(S, T(sc.X).view(-1), v0, E, steps)
    J = centroid_loss(xT, mass, body, target)
    J.backward()
    _, ck = _rollout(S, sc, steps, E=sc.E)
    frozen = [c[3] for c in ck]
    rng = np.random.default_rng(1)
    w = rng.choice([-1.0, 1.0], size=sc.n_tets)
    eps = 1e-6                                   # relative step in E, as for v0
    vals = []
    for sgn in (1, -1):
        xs, _ = _rollout(S, sc, steps, frozen, E=sc.E * (1 + sgn * eps * w))
        vals.append(float(centroid_loss(xs, mass, body, target)))
    fd = (vals[0] - vals[1]) / (2 * eps)
    adj = float((E.grad * T(sc.E) * T(w)).sum())
    assert adj == pytest.approx(fd, rel=1e-5)
    u = np.zeros_like(sc.V0)
    u[sc.body == 0] = rng.normal(size=(int((sc.body == 0).sum()), 3))
    vals = []
    for sgn in (1, -1):
        xs, _ = _rollout(S, sc, steps, frozen, E=sc.E, V0=sc.V0 + sgn * 1e-6 * u)
        vals.append(float(centroid_loss(xs, mass, body, target)))
    fd = (vals[0] - vals[1]) / 2e-6
    assert float((v0.grad * T(u).view(-1)).sum()) == pytest.approx(fd, rel=1e-5)
