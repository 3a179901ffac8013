"""Global incremental potential, BAL objective, gradient, assembled projected
Hessian and assembled stiffness Lambda, FP64 (test infrastructure).

Incremental potential (Sec. 3.1):
    E(x) = 1/(2 h^2) ||x - y||_M^2 + Psi(x),   y = x_t + h v_t + h^2 g,
with the lumped mass M. The friction potential D of Sec. 4.1 (oracle/friction)
enters every function below through the optional lagged friction set `fric`
(None = frictionless, the default).
BAL objective (Sec. 3.3, Eq. aug-lag):
    L_sigma(x) = E(x) + sigma sum_{i in A} b(d_i, dhat)
               + sum_{i in A'} [ mu_i (dhat + s_i - d_i) + sigma b(d_i, dhat + s_i) ].
Pinned vertices are Dirichlet: they stay at their initial position, their
gradient entries are zero, and their rows / columns of the Hessian are
eliminated with the diagonal block set to m_v / h^2 I (App. C, "static
boundaries"). The inertia term sums over free vertices only.

Assembled eigenvalue stiffness (Sec. 4.2.2): Lambda = sum_i S_i [lambda_i] S_i^T
where every stencil contributes the mean of its clamped eigenvalues (the trace
of its projected Hessian divided by its 3k DOFs) to each of its DOFs; the
stencils are the elements, the contact pairs and the lumped mass (m_v/h^2 per
DOF). e_j = sum of the three entries of node j; group_j = floor(log10 e_j).
"""
import dataclasses

import numpy as np
import scipy.sparse as sp

from . import contact, elastic, friction


@dataclasses.dataclass
class Model:
    scene: object
    Dm_inv: np.ndarray
    vol: np.ndarray
    mu: np.ndarray
    lam: np.ndarray
    mass: np.ndarray
    free: np.ndarray   # [N_v] bool
    h: float
    dhat: float
    gravity: np.ndarray

    @property
    def n(self):
        return self.mass.shape[0]


def make_model(scene):
    Dm_inv, vol = elastic.rest_data(scene.X, scene.tets)
    mu, lam = elastic.lame(scene.E, scene.nu)
    mass = elastic.lumped_mass(scene.X, scene.tets, scene.rho)
    return Model(scene=scene, Dm_inv=Dm_inv, vol=vol, mu=mu, lam=lam, mass=mass,
                 free=np.asarray(scene.pinned) == 0, h=float(scene.h),
                 dhat=float(scene.dhat), gravity=np.asarray(scene.gravity, dtype=np.float64))


def inertia_target(model, x_t, v_t):
    """y = x_t + h v_t + h^2 g (Sec. 3.1)."""
    return x_t + model.h * v_t + model.h ** 2 * model.gravity[None, :]


@dataclasses.dataclass
class PairSet:
    """Pairs evaluated in one objective: keys, membership in A and A', mu, s."""
    keys: list
    inA: np.ndarray
    inAp: np.ndarray
    mu: np.ndarray
    s: np.ndarray


def empty_pairs():
    z = np.zeros(0)
    return PairSet([], z.astype(bool), z.astype(bool), z, z)


def energy_parts(model, x, y, pairs: PairSet, sigma, fric=None):
    """(inertia, elastic, contact) terms of L_sigma at x; elastic is +inf if
    any tet is inverted. The contact term includes friction when fric is given."""
    sc = model.scene
    r = x - y
    inertia = 0.5 / model.h ** 2 * np.sum(model.mass[model.free] * np.sum(r[model.free] ** 2, axis=1))
    F = elastic.deformation_gradient(x, sc.tets, model.Dm_inv)
    el = float(np.sum(model.vol * elastic.psi(F, model.mu, model.lam)))
    con = 0.0
    if pairs.keys:
        e = contact.pair_energies(x, pairs.keys, sc, pairs.inA, pairs.inAp, pairs.mu, pairs.s,
                                  sigma, model.dhat)
        con = float(np.sum(e))
    con += friction.energy(fric, x)
    return float(inertia), el, con


def energy(model, x, y, pairs, sigma, fric=None):
    return float(sum(energy_parts(model, x, y, pairs, sigma, fric)))


def _scatter_vec(n_v, nodes, g):
    out = np.zeros((n_v, 3))
    for k in range(nodes.shape[1]):
        np.add.at(out, nodes[:, k], g[:, 3 * k:3 * k + 3])
    return out


def gradient(model, x, y, pairs: PairSet, sigma, parts=False, fric=None):
    """grad L_sigma [N_v,3], pinned rows zeroed. With parts=True also returns
    (inertia + elastic) gradient and the contact gradient separately."""
    sc = model.scene
    gi = model.mass[:, None] * (x - y) / model.h ** 2
    _, ge, _ = elastic.element_terms(x, sc.tets, model.Dm_inv, model.vol, model.mu,
                                     model.lam, project=False)
    gE = gi + _scatter_vec(model.n, sc.tets.astype(np.int64), ge)
    gc = np.zeros_like(gE)
    if pairs.keys:
        _, g, _, nodes, _ = contact.contact_terms(x, pairs.keys, sc, pairs.inA, pairs.inAp,
                                                  pairs.mu, pairs.s, sigma, model.dhat,
                                                  project=False)
        gc = _scatter_vec(model.n, nodes, g)
    if fric is not None and fric.nodes.shape[0]:
        _, gf, _ = friction.terms(fric, x, hessian=False)
        gc = gc + _scatter_vec(model.n, fric.nodes, gf)
    gE[~model.free] = 0.0
    gc[~model.free] = 0.0
    if parts:
        return gE + gc, gE, gc
    return gE + gc


def _coo_blocks(nodes, H, n_dof):
    """COO triplets of a batch of stencil Hessians [n,3k,3k] over nodes [n,k]."""
    n, k = nodes.shape
    dof = (3 * nodes[:, :, None] + np.arange(3)[None, None, :]).reshape(n, 3 * k)
    rows = np.broadcast_to(dof[:, :, None], (n, 3 * k, 3 * k)).ravel()
    cols = np.broadcast_to(dof[:, None, :], (n, 3 * k, 3 * k)).ravel()
    return rows, cols, H.ravel()


def hessian(model, x, y, pairs: PairSet, sigma, project=True, with_lambda=False, fric=None,
            elastic_projection="F"):
    """Assembled PSD-projected Hessian of L_sigma as scipy CSR [3N_v, 3N_v],
    pinned rows / columns eliminated with diagonal m/h^2. Friction stencils
    (PSD by construction, not projected) add their Hessians and their trace
    means to Lambda. elastic_projection: "F" (9x9 dP/dF, both paths) or
    "stencil" (12x12 element block) when project is set."""
    sc = model.scene
    nd = 3 * model.n
    _, _, He = elastic.element_terms(x, sc.tets, model.Dm_inv, model.vol, model.mu,
                                     model.lam, project=elastic_projection if project else False)
    r1, c1, v1 = _coo_blocks(sc.tets.astype(np.int64), He, nd)
    rows, cols, vals = [r1], [c1], [v1]
    lam = np.repeat(model.mass / model.h ** 2, 3)
    tr_e = np.trace(He, axis1=1, axis2=2) / 12.0
    for k in range(4):
        for a in range(3):
            np.add.at(lam, 3 * sc.tets[:, k].astype(np.int64) + a, tr_e)
    if pairs.keys:
        _, _, Hc, nodes, _ = contact.contact_terms(x, pairs.keys, sc, pairs.inA, pairs.inAp,
                                                   pairs.mu, pairs.s, sigma, model.dhat,
                                                   project=project)
        r2, c2, v2 = _coo_blocks(nodes, Hc, nd)
        rows.append(r2)
        cols.append(c2)
        vals.append(v2)
        tr_c = np.trace(Hc, axis1=1, axis2=2) / 12.0
        for k in range(4):
            for a in range(3):
                np.add.at(lam, 3 * nodes[:, k] + a, tr_c)
    if fric is not None and fric.nodes.shape[0]:
        _, _, Hf = friction.terms(fric, x)
        r3, c3, v3 = _coo_blocks(fric.nodes, Hf, nd)
        rows.append(r3)
        cols.append(c3)
        vals.append(v3)
        tr_f = np.trace(Hf, axis1=1, axis2=2) / 12.0
        for k in range(4):
            for a in range(3):
                np.add.at(lam, 3 * fric.nodes[:, k] + a, tr_f)
    dm = np.repeat(model.mass / model.h ** 2, 3)
    rows.append(np.arange(nd))
    cols.append(np.arange(nd))
    vals.append(dm)
    H = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nd, nd)).tocsr()
    H.sum_duplicates()
    pinned_dof = np.repeat(~model.free, 3)
    if pinned_dof.any():
        keep = sp.diags((~pinned_dof).astype(np.float64))
        H = (keep @ H @ keep).tocsr()
        H = H + sp.diags(np.where(pinned_dof, dm, 0.0))
        H = H.tocsr()
    if with_lambda:
        return H, lam
    return H


def groups_from_lambda(lam):
    """e_j = sum of node j's three Lambda entries; group = floor(log10 e_j)."""
    e = lam.reshape(-1, 3).sum(axis=1)
    return e, np.floor(np.log10(e)).astype(np.int64)


def masked_hessian(H, groups):
    """H_dom of the warm start (Sec. 4.2.2): the assembled Hessian without the
    entries that couple nodes of different stiffness groups."""
    H = H.tocoo()
    g = np.asarray(groups)
    keep = g[H.row // 3] == g[H.col // 3]
    return sp.coo_matrix((H.data[keep], (H.row[keep], H.col[keep])), shape=H.shape).tocsr()
