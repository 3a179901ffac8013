"""Neo-Hookean tetrahedral elasticity, FP64 (test infrastructure).

The paper names the material model only ("Neo-Hookean", Sec. 1 and Sec. 6.2)
and never writes Psi. Reading used throughout (the NH of IPC):

    Psi(F) = mu/2 (tr(F^T F) - 3) - mu ln J + lam/2 (ln J)^2,   J = det F,
    mu = E / (2 (1 + nu)),  lam = E nu / ((1 + nu)(1 - 2 nu)),
    Psi = +inf for J <= 0 (inverted elements are rejected by the line search).

Per tet e with rest edge matrix D_m = [X1-X0, X2-X0, X3-X0] and rest volume
V_e = |det D_m| / 6: F = D_s D_m^{-1}, W_e = V_e Psi(F). The element stencil
Hessian is projected to PSD in deformation-gradient space: the 9x9 dP/dF is
eigen-decomposed, negative eigenvalues are set to zero, and the 12x12 element
block is V_e G^T Proj(dP/dF) G, G = d vec(F) / d x (Sec. 4.2.2 "stencil-wise
eigendecomposition ... closest symmetric positive semi-definite form"; the
9x9 reading is listed in the design notes).

Vectorisation conventions: vec(F) index = 3*i + j for F[i, j]; the 12 element
DOFs are ordered (vertex a, axis k) -> 3*a + k.
"""
import numpy as np


def lame(E, nu):
    E = np.asarray(E, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def rest_data(X, tets):
    """D_m^{-1} [N_t,3,3] and rest volumes V [N_t]."""
    X = np.asarray(X, dtype=np.float64)
    t = np.asarray(tets, dtype=np.int64)
    Dm = np.stack([X[t[:, 1]] - X[t[:, 0]], X[t[:, 2]] - X[t[:, 0]],
                   X[t[:, 3]] - X[t[:, 0]]], axis=2)  # columns are edges
    vol = np.abs(np.linalg.det(Dm)) / 6.0
    return np.linalg.inv(Dm), vol


def lumped_mass(X, tets, rho):
    """Lumped (diagonal) mass, Sec. 3.1: each tet gives rho V_e / 4 to each of
    its four vertices."""
    _, vol = rest_data(X, tets)
    m = np.zeros(np.asarray(X).shape[0])
    share = np.asarray(rho, dtype=np.float64) * vol / 4.0
    for k in range(4):
        np.add.at(m, np.asarray(tets)[:, k], share)
    return m


def shape_matrix(Dm_inv):
    """B [N_t,4,3] with dF_ij/dx_{a,k} = delta_ik B[a, j]."""
    B = np.empty(Dm_inv.shape[:-2] + (4, 3))
    B[..., 1:, :] = Dm_inv
    B[..., 0, :] = -Dm_inv.sum(axis=-2)
    return B


def grad_map(Dm_inv):
    """G [N_t,9,12] = d vec(F) / d x."""
    B = shape_matrix(Dm_inv)
    n = B.shape[0]
    G = np.zeros((n, 9, 12))
    for i in range(3):
        for j in range(3):
            for a in range(4):
                G[:, 3 * i + j, 3 * a + i] = B[:, a, j]
    return G


def deformation_gradient(x, tets, Dm_inv):
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(tets, dtype=np.int64)
    Ds = np.stack([x[t[:, 1]] - x[t[:, 0]], x[t[:, 2]] - x[t[:, 0]],
                   x[t[:, 3]] - x[t[:, 0]]], axis=2)
    return Ds @ Dm_inv


def psi(F, mu, lam):
    J = np.linalg.det(F)
    out = np.full(J.shape, np.inf)
    ok = J > 0
    Fo = F[ok]
    lnJ = np.log(J[ok])
    I1 = np.einsum("nij,nij->n", Fo, Fo)
    out[ok] = 0.5 * mu[ok] * (I1 - 3.0) - mu[ok] * lnJ + 0.5 * lam[ok] * lnJ ** 2
    return out


def first_piola(F, mu, lam):
    """P = dPsi/dF = mu (F - F^{-T}) + lam ln J F^{-T}."""
    J = np.linalg.det(F)
    FinvT = np.swapaxes(np.linalg.inv(F), -1, -2)
    lnJ = np.log(J)
    return mu[:, None, None] * (F - FinvT) + (lam * lnJ)[:, None, None] * FinvT


def dPdF(F, mu, lam):
    """9x9 d vec(P) / d vec(F).

    With A = F^{-T}: d A_ij / d F_kl = -A_il A_kj and d ln J / d F_kl = A_kl, so
    dP_ij/dF_kl = mu d_ik d_jl + (mu - lam ln J) A_il A_kj + lam A_ij A_kl.
    """
    J = np.linalg.det(F)
    A = np.swapaxes(np.linalg.inv(F), -1, -2)
    lnJ = np.log(J)
    eye = np.eye(3)
    T = (mu[:, None, None, None, None] * np.einsum("ik,jl->ijkl", eye, eye)[None]
         + (mu - lam * lnJ)[:, None, None, None, None] * np.einsum("nil,nkj->nijkl", A, A)
         + lam[:, None, None, None, None] * np.einsum("nij,nkl->nijkl", A, A))
    return T.reshape(-1, 9, 9)


def project_psd(H):
    """Nearest symmetric PSD matrix in the Frobenius norm: eigen-decompose and
    set negative eigenvalues to zero (batched over the leading axes)."""
    Hs = 0.5 * (H + np.swapaxes(H, -1, -2))
    w, V = np.linalg.eigh(Hs)
    w = np.maximum(w, 0.0)
    return np.einsum("...ik,...k,...jk->...ij", V, w, V)


def element_terms(x, tets, Dm_inv, vol, mu, lam, project=True):
    """Per-tet energy W_e [N_t], gradient [N_t,12] and Hessian [N_t,12,12].
    project: False (exact Hessian), True or "F" (PSD projection of the 9x9
    dP/dF, the reading used by both paths), or "stencil" (the nearest PSD
    matrix to the 12x12 element block V_e G^T (dP/dF) G itself, the other
    reading of Sec. 4.2.2, kept to measure the difference)."""
    F = deformation_gradient(x, tets, Dm_inv)
    W = vol * psi(F, mu, lam)
    P = first_piola(F, mu, lam)
    G = grad_map(Dm_inv)
    g = vol[:, None] * np.einsum("nab,na->nb", G, P.reshape(-1, 9))
    K = dPdF(F, mu, lam)
    if project is True or project == "F":
        K = project_psd(K)
    H = vol[:, None, None] * np.einsum("nai,nab,nbj->nij", G, K, G)
    if project == "stencil":
        H = project_psd(H)
    return W, g, H
