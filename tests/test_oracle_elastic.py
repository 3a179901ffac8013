"""Pins for the Neo-Hookean element terms and the PSD projection."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import elastic
from paper_2407_00046_b300 import scenes


def rand_F(rng, n, jmin=0.5, jmax=2.0):
    out = []
    while len(out) < n:
        F = np.eye(3) + 0.35 * rng.normal(size=(3, 3))
        J = np.linalg.det(F)
        if jmin <= J <= jmax:
            out.append(F)
    return np.array(out)


def test_rest_state_is_stress_free():
    F = np.tile(np.eye(3), (3, 1, 1))
    mu, lam = elastic.lame(np.array([1e5, 1e6, 1e9]), np.array([0.4, 0.3, 0.45]))
    assert np.all(elastic.psi(F, mu, lam) == 0)
    assert np.abs(elastic.first_piola(F, mu, lam)).max() == 0


def test_rest_tangent_is_linear_elasticity():
    # at F = I, dP/dF = mu (d_ik d_jl + d_il d_jk) + lam d_ij d_kl (textbook)
    mu, lam = elastic.lame(np.array([3e5]), np.array([0.4]))
    K = elastic.dPdF(np.eye(3)[None], mu, lam)[0].reshape(3, 3, 3, 3)
    I = np.eye(3)
    C = (mu[0] * (np.einsum("ik,jl->ijkl", I, I) + np.einsum("il,jk->ijkl", I, I))
         + lam[0] * np.einsum("ij,kl->ijkl", I, I))
    assert np.allclose(K, C, rtol=1e-14, atol=1e-9)
    # Lame constants from E, nu (textbook): E = mu (3 lam + 2 mu) / (lam + mu)
    assert mu[0] * (3 * lam[0] + 2 * mu[0]) / (lam[0] + mu[0]) == pytest.approx(3e5, rel=1e-14)


def test_rotation_invariance(rng):
    F = rand_F(rng, 20)
    mu, lam = elastic.lame(np.full(20, 1e5), np.full(20, 0.4))
    R = np.array([sla.expm(np.cross(np.eye(3), rng.normal(size=3))) for _ in range(20)])
    assert np.allclose(elastic.psi(R @ F, mu, lam), elastic.psi(F, mu, lam), rtol=1e-12)


def test_piola_and_tangent_fd(rng):
    F = rand_F(rng, 10)
    mu, lam = elastic.lame(np.full(10, 2e5), np.full(10, 0.4))
    P = elastic.first_piola(F, mu, lam)
    K = elastic.dPdF(F, mu, lam)
    h = 1e-6
    for a in range(9):
        dF = np.zeros((3, 3))
        dF.flat[a] = h
        fd = (elastic.psi(F + dF, mu, lam) - elastic.psi(F - dF, mu, lam)) / (2 * h)
        assert np.allclose(P.reshape(-1, 9)[:, a], fd, rtol=1e-6, atol=1e-3)
        fdP = (elastic.first_piola(F + dF, mu, lam) - elastic.first_piola(F - dF, mu, lam)) / (2 * h)
        assert np.allclose(K[:, :, a], fdP.reshape(-1, 9), rtol=1e-6, atol=1e-3)
    assert np.allclose(K, np.swapaxes(K, 1, 2), rtol=1e-13, atol=1e-6)


def _one_tet(rng):
    X = np.array([[0, 0, 0], [0.01, 0, 0], [0, 0.012, 0], [0.001, 0.002, 0.011]], float)
    tets = np.array([[0, 1, 2, 3]])
    Dm_inv, vol = elastic.rest_data(X, tets)
    x = X + 0.002 * rng.normal(size=X.shape)
    mu, lam = elastic.lame(np.array([1e5]), np.array([0.4]))
    return X, x, tets, Dm_inv, vol, mu, lam


def test_element_gradient_hessian_fd(rng):
    for _ in range(5):
        X, x, tets, Dm_inv, vol, mu, lam = _one_tet(rng)
        W, g, H = elastic.element_terms(x, tets, Dm_inv, vol, mu, lam, project=False)
        h = 1e-8
        for a in range(12):
            dx = np.zeros(12)
            dx[a] = h
            xp, xm = x + dx.reshape(4, 3), x - dx.reshape(4, 3)
            Wp, gp, _ = elastic.element_terms(xp, tets, Dm_inv, vol, mu, lam, project=False)
            Wm, gm, _ = elastic.element_terms(xm, tets, Dm_inv, vol, mu, lam, project=False)
            assert g[0, a] == pytest.approx((Wp[0] - Wm[0]) / (2 * h), rel=1e-5, abs=1e-9)
            assert np.allclose(H[0, :, a], (gp[0] - gm[0]) / (2 * h), rtol=1e-5, atol=1e-6)
        # volume is |det Dm| / 6
        assert vol[0] == pytest.approx(abs(np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], 1))) / 6)


def test_projection_is_nearest_psd(rng):
    for n in (9, 12):
        A = rng.normal(size=(20, n, n))
        A = A + np.swapaxes(A, 1, 2)
        P = elastic.project_psd(A)
        assert np.allclose(P, np.swapaxes(P, 1, 2), atol=1e-13)
        assert np.linalg.eigvalsh(P).min() > -1e-12 * np.abs(P).max()
        assert np.allclose(elastic.project_psd(P), P, atol=1e-12)
        # independent construction: (A + |A|)/2 with |A| = sqrtm(A^2) (polar factor)
        for k in range(5):
            Q = 0.5 * (A[k] + np.real(sla.sqrtm(A[k] @ A[k])))
            assert np.allclose(P[k], Q, atol=1e-9)


def test_projected_element_hessian_is_psd_and_translation_invariant(rng):
    X, _, tets, Dm_inv, vol, mu, lam = _one_tet(rng)
    for _ in range(5):
        x = X + 0.004 * rng.normal(size=X.shape)
        _, _, H = elastic.element_terms(x, tets, Dm_inv, vol, mu, lam, project=True)
        assert np.linalg.eigvalsh(H[0]).min() > -1e-9 * np.abs(H).max()
        # rigid translations are in the null space (row sums over vertices vanish)
        assert np.abs(H[0].reshape(12, 4, 3).sum(axis=1)).max() < 1e-9 * np.abs(H).max()


def test_lumped_mass_and_volume():
    X, T = scenes.lattice_box(3, 2, 4, (0.3, 0.2, 0.4))
    _, vol = elastic.rest_data(X, T)
    assert vol.sum() == pytest.approx(0.3 * 0.2 * 0.4, rel=1e-13)
    m = elastic.lumped_mass(X, T, np.full(T.shape[0], 1000.0))
    assert m.sum() == pytest.approx(1000 * 0.3 * 0.2 * 0.4, rel=1e-13)
