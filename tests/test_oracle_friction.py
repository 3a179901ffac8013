"""Pins for the fully-implicit friction of Sec. 4.1 (oracle/friction): the
mollifier's branches, the closest-point weights against brute force, finite
differences of the friction gradient and Hessian in the static and sliding
zones, PSD without projection, and Coulomb's law on a sliding cube."""
import numpy as np
import pytest

from oracle import bal, distance, friction, system
from paper_2407_00046_b300 import scenes


def test_mollifier_branches_join_c2():
    eh = 3e-5
    for side in (eh * (1 - 1e-12), eh * (1 + 1e-12)):
        f, f1, f2 = friction.mollifier(np.array([side]), eh)
        assert abs(f[0] - 2 * eh / 3) < 1e-10 * eh
        assert abs(f1[0] - 1.0) < 1e-10
        assert abs(f2[0]) < 1e-6 / eh
    f, f1, f2 = friction.mollifier(np.array([0.0]), eh)
    assert f[0] == 0 and f1[0] == 0 and f2[0] == pytest.approx(2 / eh)
    # monotone and convex
    y = np.linspace(0, 3 * eh, 301)
    f, f1, f2 = friction.mollifier(y, eh)
    assert np.all(np.diff(f) > 0) and np.all(f1 >= 0) and np.all(f2 >= 0)


def _random_stencils(rng, n, ee):
    X4 = rng.normal(size=(n, 4, 3))
    X4[:, 2:] += rng.normal(size=(n, 1, 3)) * 0.7 if ee else 0.0
    return X4


def _brute_closest(X, ee, m=161):
    """Closest points by dense sampling of both primitives."""
    s = np.linspace(0, 1, m)
    if ee:
        A = X[0][None] + s[:, None] * (X[1] - X[0])[None]
        B = X[2][None] + s[:, None] * (X[3] - X[2])[None]
        D = np.linalg.norm(A[:, None] - B[None], axis=2)
        i, j = np.unravel_index(np.argmin(D), D.shape)
        return D[i, j], A[i] - B[j]
    u, v = np.meshgrid(s, s, indexing="ij")
    keep = u + v <= 1
    u, v = u[keep], v[keep]
    Q = X[1][None] + u[:, None] * (X[2] - X[1])[None] + v[:, None] * (X[3] - X[1])[None]
    D = np.linalg.norm(X[0][None] - Q, axis=1)
    k = np.argmin(D)
    return D[k], X[0] - Q[k]


@pytest.mark.parametrize("ee", [False, True])
def test_closest_weights_give_the_closest_points(ee):
    rng = np.random.default_rng(7 if ee else 8)
    X4 = _random_stencils(rng, 40, ee)
    regions = distance.classify(X4, np.full(40, ee))
    d = distance.distances(X4, regions)
    beta = friction.closest_weights(X4, regions)
    kinds = {r[0] for r in regions}
    assert len(kinds) >= 2                      # interior and degenerate regions both covered
    for i in range(40):
        nvec = beta[i] @ X4[i]
        assert abs(np.linalg.norm(nvec) - d[i]) < 1e-12 * max(1.0, d[i])
        first, second = (beta[i][:2], beta[i][2:]) if ee else (beta[i][:1], beta[i][1:])
        assert abs(first.sum() - 1) < 1e-12 and abs(second.sum() + 1) < 1e-12
        assert first.min() >= -1e-12 and second.max() <= 1e-12     # convex combinations
        db, vb = _brute_closest(X4[i], ee)
        assert db >= d[i] - 1e-12                                  # nothing closer exists
        assert np.linalg.norm(vb - nvec) < 0.05 * max(1.0, np.linalg.norm(X4[i]).max())


def _fset(rng, n, eh, scale):
    X4 = _random_stencils(rng, n, True)
    regions = distance.classify(X4, np.ones(n, bool))
    x = X4.reshape(-1, 3)
    nodes = np.arange(4 * n).reshape(n, 4)
    lam = rng.uniform(0.5, 2.0, n)
    x_t = x - scale * rng.normal(size=x.shape)
    return friction.lag(x, x_t, nodes, regions, lam, 0.4, eh), x


@pytest.mark.parametrize("zone,scale", [("static", 1e-6), ("sliding", 1e-3)])
def test_friction_gradient_and_hessian_match_finite_differences(zone, scale):
    rng = np.random.default_rng(11)
    eh = 3e-5
    fs, x = _fset(rng, 6, eh, scale)
    w, _ = friction._tangent(fs, x)
    y = np.linalg.norm(w, axis=1)
    assert np.all(y < eh) if zone == "static" else np.all(y > eh)
    e, g, H = friction.terms(fs, x)
    for j in range(fs.nodes.shape[0]):
        sub = friction.FrictionSet(fs.nodes[j:j + 1], fs.beta[j:j + 1], fs.normal[j:j + 1],
                                   fs.lam[j:j + 1], fs.chi, fs.eps_h, fs.x_t)
        x0 = x.copy()
        idx = fs.nodes[j]
        step = 1e-3 * max(y[j], 1e-12)   # O(1) coordinates: keep the step well above their rounding
        gfd = np.zeros(12)
        Hfd = np.zeros((12, 12))
        for k in range(12):
            xp, xm = x0.copy(), x0.copy()
            xp[idx[k // 3], k % 3] += step
            xm[idx[k // 3], k % 3] -= step
            gfd[k] = (friction.energy(sub, xp) - friction.energy(sub, xm)) / (2 * step)
            gp = friction.terms(sub, xp, hessian=False)[1][0]
            gm = friction.terms(sub, xm, hessian=False)[1][0]
            Hfd[:, k] = (gp - gm) / (2 * step)
        assert np.abs(gfd - g[j]).max() < 1e-5 * np.abs(g[j]).max()
        assert np.abs(Hfd - H[j]).max() < 1e-4 * np.abs(H[j]).max()


def test_friction_hessian_is_psd_without_projection():
    rng = np.random.default_rng(12)
    for scale in (0.0, 1e-6, 3e-5, 1e-3):
        fs, x = _fset(rng, 20, 3e-5, scale)
        _, _, H = friction.terms(fs, x)
        ev = np.linalg.eigvalsh(H)
        assert ev.min() >= -1e-9 * np.abs(ev).max()


def test_sliding_friction_force_is_coulomb():
    """Beyond eps h the force on each primitive has magnitude chi lambda,
    along the tangent slip direction, whatever the slip length."""
    rng = np.random.default_rng(13)
    fs, x = _fset(rng, 10, 3e-5, 1e-2)
    w, _ = friction._tangent(fs, x)
    _, g, _ = friction.terms(fs, x, hessian=False)
    G = g.reshape(-1, 4, 3)
    F1 = G[:, :2].sum(axis=1)                      # first edge's share
    assert np.allclose(np.linalg.norm(F1, axis=1), fs.chi * fs.lam, rtol=1e-12)
    what = w / np.linalg.norm(w, axis=1)[:, None]
    assert np.allclose(F1, (fs.chi * fs.lam)[:, None] * what, rtol=1e-10, atol=1e-14)
    assert np.abs(G.sum(axis=1)).max() < 1e-14     # equal and opposite


@pytest.mark.parametrize("chi", [0.0, 0.3])
def test_coulomb_law_on_a_sliding_cube(chi):
    """Momentum balance of the converged backward-Euler step: the cube's
    tangential impulse is chi times its normal impulse (Coulomb) while it
    slides, and zero without friction."""
    sc = scenes.sliding_cube()
    m = system.make_model(sc)
    c = sc.body == 0
    M = m.mass[c].sum()
    t_dir = np.array([1.0, 0.0, 1.0]) / np.sqrt(2.0)
    x, v = sc.X.copy(), sc.V0.copy()
    for _ in range(2):
        vb = (m.mass[c, None] * v[c]).sum(axis=0) / M
        x, v, info = bal.time_step(m, x, v, bal.Params(newton_tol=1e-9, friction=chi, newton_max=300))
        assert info["converged"]
        va = (m.mass[c, None] * v[c]).sum(axis=0) / M
        dv = va - vb
        ratio = -(dv @ t_dir) / (dv[1] - sc.gravity[1] * sc.h)
        assert abs(ratio - chi) < 1e-5
        assert va @ t_dir > 0.3                    # still sliding
