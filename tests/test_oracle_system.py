"""Pins for the global objective, gradient, assembled Hessian, contact terms
and the assembled stiffness Lambda."""
import copy

import numpy as np
import pytest

from oracle import barrier, bal, contact, distance, system
from paper_2407_00046_b300 import scenes


@pytest.fixture(scope="module")
def close_cubes():
    sc = scenes.two_cubes(n=2)
    m = system.make_model(sc)
    x = sc.X.copy()
    x[sc.body == 1, 1] -= 0.01 - 0.0004      # top cube 0.4 mm above
    x[sc.body == 1, 0] += 0.013               # misalign the lattices
    return sc, m, x


def test_candidate_pairs_superset_brute_force(close_cubes):
    sc, m, x = close_cubes
    r = 2e-3
    cand = set(contact.candidate_pairs(x, sc, r))
    allp = [(0, int(v), int(t)) for v in sc.surf_verts for t in range(len(sc.tris))
            if v not in sc.tris[t]]
    E = sc.edges
    allp += [(1, a, b) for a in range(len(E)) for b in range(a + 1, len(E))
             if not set(E[a]) & set(E[b])]
    d, _, _ = contact.pair_distances(x, allp, sc)
    close = {k for k, dd in zip(allp, d) if dd < r}
    assert close and close <= cand


def _pairset(m, x, keys, Ap_mu):
    ps = bal.make_pairset(m, x, keys, Ap_mu, 3.0)
    return ps


def test_global_gradient_and_hessian_fd(close_cubes):
    sc, m, x = close_cubes
    rng = np.random.default_rng(5)
    x = x + 2e-5 * rng.normal(size=x.shape) * (sc.pinned == 0)[:, None]
    y = system.inertia_target(m, sc.X, sc.V0)
    keys, d = bal.active_pairs(m, x)
    assert len(keys) > 10
    Ap = {k: 0.7 for k in keys[::3]}
    ps = _pairset(m, x, keys, Ap)
    sigma = 3.0
    g = system.gradient(m, x, y, ps, sigma).ravel()
    H = system.hessian(m, x, y, ps, sigma, project=False).toarray()
    free = np.repeat(sc.pinned == 0, 3)
    h = 1e-9
    idx = np.flatnonzero(free)[rng.choice(free.sum(), 12, replace=False)]
    for a in idx:
        dx = np.zeros(x.size)
        dx[a] = h
        Ep = system.energy(m, x + dx.reshape(-1, 3), y, ps, sigma)
        Em = system.energy(m, x - dx.reshape(-1, 3), y, ps, sigma)
        assert g[a] == pytest.approx((Ep - Em) / (2 * h), rel=2e-5, abs=1e-6)
        gp = system.gradient(m, x + dx.reshape(-1, 3), y, ps, sigma).ravel()
        gm = system.gradient(m, x - dx.reshape(-1, 3), y, ps, sigma).ravel()
        fd = (gp - gm) / (2 * h)
        assert np.allclose(H[free, a], fd[free], rtol=1e-4, atol=1e-3 * np.abs(H[:, a]).max())
    assert np.allclose(H, H.T, atol=1e-9 * np.abs(H).max())


def test_projected_hessian_psd_and_pins(close_cubes):
    sc, m, x = close_cubes
    y = system.inertia_target(m, sc.X, sc.V0)
    keys, _ = bal.active_pairs(m, x)
    ps = _pairset(m, x, keys, {})
    H, lam = system.hessian(m, x, y, ps, 5.0, with_lambda=True)
    Hd = H.toarray()
    assert np.linalg.eigvalsh(Hd).min() > 0
    pin = np.repeat(sc.pinned == 1, 3)
    sub = Hd[pin]
    assert np.allclose(sub[:, ~pin], 0) and np.allclose(np.diag(Hd)[pin], np.repeat(m.mass / m.h ** 2, 3)[pin])
    # Lambda: mass term + mean clamped eigenvalue of each stencil per DOF
    assert np.all(lam >= np.repeat(m.mass / m.h ** 2, 3) * (1 - 1e-12))
    e, grp = system.groups_from_lambda(lam)
    assert np.all(grp == np.floor(np.log10(e)))


def test_elastic_hessian_row_sums_vanish_at_rest():
    sc = scenes.two_cubes(n=2)
    sc.pinned[:] = 0
    m = system.make_model(sc)
    y = sc.X
    H = system.hessian(m, sc.X, y, system.empty_pairs(), 1.0).toarray()
    H -= np.diag(np.repeat(m.mass / m.h ** 2, 3))
    T = np.zeros((sc.n_verts * 3, 3))
    for a in range(3):
        T[a::3, a] = 1
    assert np.abs(H @ T).max() < 1e-9 * np.abs(H).max()


def test_al_gradient_closed_form_with_zero_slack(rng):
    # with s = 0 the augmentation gradient is (-mu + sigma b'(d, dhat)) grad d
    X4 = rng.normal(size=(4, 3)) * 1e-3
    reg = distance.classify(X4[None], [False])
    d, gd, _ = distance.distance_derivatives(X4[None], reg)
    dh = 2.0 * d[0]
    e, e1, e2 = contact.phi_derivs(d, [0.0], [1.0], np.array([0.3]), np.array([0.0]), 7.0, dh)
    assert e1[0] == pytest.approx(-0.3 + 7.0 * barrier.db(d, dh)[0], rel=1e-15)
    assert e[0] == pytest.approx(0.3 * (dh - d[0]) + 7.0 * barrier.b(d, dh)[0], rel=1e-15)


def test_slack_elimination_closed_form():
    # s = max(-mu/sigma - dhat + d, 0) minimises mu c + sigma/2 c^2, c = dhat + s - d
    mu, sigma, dh = 0.4, 50.0, 1e-3
    for d in (2e-4, 9e-4, 1.2e-3, 5e-3):
        s_grid = np.linspace(0, 0.01, 200001)
        c = dh + s_grid - d
        s_bf = s_grid[np.argmin(mu * c + 0.5 * sigma * c ** 2)]
        s_cf = max(-mu / sigma - dh + d, 0.0)
        assert abs(s_bf - s_cf) <= 1e-7


def test_lambda_is_the_mean_clamped_eigenvalue_of_every_stencil(close_cubes):
    """Lambda (Sec. 4.2.2) from eigenvalues rather than traces: every element,
    contact pair and friction stencil adds the mean of the eigenvalues of its
    projected Hessian to each of its 12 DOFs, on top of m / h^2."""
    from oracle import elastic, friction
    sc, m, x = close_cubes
    rng = np.random.default_rng(31)
    xd = x + 1e-4 * rng.normal(size=x.shape) * (sc.pinned == 0)[:, None]
    y = system.inertia_target(m, sc.X, sc.V0)
    keys, _ = bal.active_pairs(m, xd)
    assert keys
    ps = _pairset(m, xd, keys, {})
    fs = bal.friction_set(m, xd, x, ps, 5.0, bal.Params(friction=0.4))
    _, lam = system.hessian(m, xd, y, ps, 5.0, with_lambda=True, fric=fs)
    ref = np.repeat(m.mass / m.h ** 2, 3)

    def add(nodes, H):
        mean = np.linalg.eigvalsh(H).mean(axis=1)
        for k in range(4):
            for a in range(3):
                np.add.at(ref, 3 * nodes[:, k] + a, mean)

    _, _, He = elastic.element_terms(xd, sc.tets, m.Dm_inv, m.vol, m.mu, m.lam, project=True)
    add(sc.tets.astype(np.int64), He)
    _, _, Hc, nodes, _ = contact.contact_terms(xd, ps.keys, sc, ps.inA, ps.inAp, ps.mu, ps.s, 5.0, m.dhat)
    add(nodes, Hc)
    add(fs.nodes, friction.terms(fs, xd)[2])
    assert np.abs(lam - ref).max() <= 1e-12 * np.abs(ref).max()


def test_block_rows_sum_to_the_mass_term_away_from_pins(close_cubes):
    """Translation invariance of every projected stencil Hessian (elastic,
    contact with A and A', friction): away from pinned vertices the 3x3
    blocks of a row of H sum to m_i/h^2 I, the property the difference form
    of the FP32 operator relies on; rows next to a pinned vertex differ by the
    blocks dropped with it."""
    sc, m, x = close_cubes
    rng = np.random.default_rng(3)
    xd = x + 2e-5 * rng.normal(size=x.shape) * (sc.pinned == 0)[:, None]
    y = system.inertia_target(m, sc.X, sc.V0)
    keys, d = bal.active_pairs(m, xd)
    assert len(keys) > 4
    Ap_mu = {keys[k]: 0.5 + k for k in range(0, len(keys), 3)}     # some pairs also in A'
    ps = bal.make_pairset(m, xd, keys, Ap_mu, 3.0)
    assert ps.inAp.any()
    fric = bal.friction_set(m, xd, x, ps, 3.0, bal.Params(friction=0.3))
    assert fric is not None
    H = system.hessian(m, xd, y, ps, 3.0, fric=fric).toarray()
    n = sc.n_verts
    T = np.zeros((3 * n, 3))
    for a in range(3):
        T[a::3, a] = 1
    rows = (H @ T).reshape(n, 3, 3)                  # block-row sums
    pinned = sc.pinned == 1
    # stencil adjacency from the same system with nothing pinned (pinning
    # zeroes the blocks between a free and a pinned vertex)
    sc_free = copy.deepcopy(sc)
    sc_free.pinned[:] = 0
    m_free = system.make_model(sc_free)
    H_free = system.hessian(m_free, xd, y, ps, 3.0, fric=fric).toarray()
    Hb = np.abs(H_free).reshape(n, 3, n, 3).max(axis=(1, 3))
    near_pin = (Hb[:, pinned] > 0).any(axis=1) & ~pinned
    interior = ~pinned & ~near_pin
    expect = (m.mass / m.h ** 2)[:, None, None] * np.eye(3)[None]
    assert interior.sum() > n // 4 and near_pin.any()
    assert np.abs(rows[interior] - expect[interior]).max() < 1e-9 * np.abs(H).max()
    # with nothing pinned every row sums to its mass term
    rows_free = (H_free @ T).reshape(n, 3, 3)
    assert np.abs(rows_free - expect).max() < 1e-9 * np.abs(H_free).max()
