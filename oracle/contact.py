"""Contact pairs and their barrier / augmented-Lagrangian terms, FP64
(test infrastructure).

Constraint set (Sec. 3.1, Eq. problem): every point-triangle pair (surface
vertex v, surface triangle t, v not a vertex of t) and every edge-edge pair
(surface edges e < f sharing no vertex) whose unsigned distance is below the
offset dhat is active (the set A). Pairs are identified by
(kind, first id, second id) with kind 0 = PT (vertex id, triangle index) and
kind 1 = EE (edge index, edge index).

Per pair i the energy of Eq. (aug-lag) is a function of d_i only:

    phi_i(d) = [i in A] sigma b(d, dhat)
             + [i in A'] ( mu_i (dhat + s_i - d) + sigma b(d, dhat + s_i) ),

so grad = phi' grad d and Hessian = phi'' grad d grad d^T + phi' Hess d; the
12x12 stencil Hessian is then projected to the nearest PSD matrix
(Sec. 4.2.2). s_i (Sec. 3.2.2) is held fixed inside an iteration.

Edge-edge pairs are mollified (reading: the paper takes its contact potential
from IPC and is silent on parallel edges; IPC, Li et al. 2020, Sec. 4.3, scales
every edge-edge term by a mollifier because the segment-segment distance is
not C^1 where the edges become parallel):

    phi_EE(x) = m(c) phi(d),  c = |u x v|^2  (u, v the two edge vectors),
    m(c) = (2 - c/eps_x) c/eps_x for c < eps_x, else 1,
    eps_x = 1e-3 |u_rest|^2 |v_rest|^2,

so grad = m phi' grad d + phi grad m and
Hessian = m (phi'' grad d grad d^T + phi' Hess d)
          + phi' (grad d grad m^T + grad m grad d^T) + phi Hess m,
projected as one 12x12 block. Derivatives of m are taken by automatic
differentiation of m(c(x)).
"""
import numpy as np
import torch
from scipy.spatial import cKDTree
from torch.func import grad, hessian, vmap

from . import barrier, distance
from .elastic import project_psd


def _pt_candidates(x, surf_verts, tris, r):
    P = x[surf_verts]
    T = x[tris]
    c = T.mean(axis=1)
    rad = np.sqrt(((T - c[:, None, :]) ** 2).sum(-1)).max(axis=1)
    tree_t = cKDTree(c)
    tree_p = cKDTree(P)
    sm = tree_p.sparse_distance_matrix(tree_t, r + rad.max() + 1e-15, output_type="ndarray")
    if sm.size == 0:
        return []
    iv, it = sm["i"].astype(np.int64), sm["j"].astype(np.int64)
    keep = sm["v"] <= r + rad[it] + 1e-15
    iv, it = iv[keep], it[keep]
    v = surf_verts[iv].astype(np.int64)
    keep = ~np.any(tris[it] == v[:, None], axis=1)
    return list(zip([0] * int(keep.sum()), v[keep].tolist(), it[keep].tolist()))


def _ee_candidates(x, edges, r):
    S = x[edges]
    c = S.mean(axis=1)
    rad = 0.5 * np.sqrt(((S[:, 1] - S[:, 0]) ** 2).sum(-1))
    tree = cKDTree(c)
    pairs = tree.query_pairs(r + 2 * rad.max() + 1e-15, output_type="ndarray")
    if pairs.size == 0:
        return []
    e, f = pairs.min(axis=1), pairs.max(axis=1)
    keep = np.sqrt(((c[e] - c[f]) ** 2).sum(-1)) <= r + rad[e] + rad[f] + 1e-15
    e, f = e[keep], f[keep]
    share = np.any(edges[e][:, :, None] == edges[f][:, None, :], axis=(1, 2))
    e, f = e[~share], f[~share]
    return [(1, int(a), int(b)) for a, b in zip(e, f)]


def candidate_pairs(x, scene, r):
    """All PT / EE pairs whose primitives' bounding spheres come within r of
    each other (a superset of the pairs with d < r), sorted by key."""
    pairs = _pt_candidates(x, scene.surf_verts, scene.tris, r) + \
        _ee_candidates(x, scene.edges, r)
    pairs.sort()
    return pairs


def stencil_nodes(pairs, scene):
    """[n,4] vertex ids of each pair's stencil."""
    if not len(pairs):
        return np.zeros((0, 4), dtype=np.int64)
    P = np.asarray(pairs, dtype=np.int64).reshape(-1, 3)
    out = np.zeros((P.shape[0], 4), dtype=np.int64)
    pt = P[:, 0] == 0
    out[pt, 0] = P[pt, 1]
    out[pt, 1:] = scene.tris[P[pt, 2]]
    ee = ~pt
    out[ee, :2] = scene.edges[P[ee, 1]]
    out[ee, 2:] = scene.edges[P[ee, 2]]
    return out


def pair_distances(x, pairs, scene):
    """Unsigned distance and region of every pair at x."""
    if not pairs:
        return np.zeros(0), [], np.zeros((0, 4), dtype=np.int64)
    nodes = stencil_nodes(pairs, scene)
    X4 = x[nodes]
    is_ee = np.asarray(pairs, dtype=np.int64).reshape(-1, 3)[:, 0] == 1
    regions = distance.classify(X4, is_ee)
    return distance.distances(X4, regions), regions, nodes


def phi_derivs(d, inA, inAp, mu, s, sigma, dhat):
    """phi, phi', phi'' of the per-pair energy (vectorised over pairs)."""
    inA = np.asarray(inA, dtype=np.float64)
    inAp = np.asarray(inAp, dtype=np.float64)
    c2 = dhat + np.asarray(s, dtype=np.float64)
    e = inA * sigma * barrier.b(d, dhat) + inAp * (mu * (c2 - d) + sigma * barrier.b(d, c2))
    e1 = inA * sigma * barrier.db(d, dhat) + inAp * (-mu + sigma * barrier.db(d, c2))
    e2 = inA * sigma * barrier.d2b(d, dhat) + inAp * sigma * barrier.d2b(d, c2)
    return e, e1, e2


MOLLIFIER_EPS = 1e-3    # eps_x = 1e-3 |u_rest|^2 |v_rest|^2 (IPC)
MOLLIFY_EE = True


def ee_eps(pairs, scene):
    """eps_x of every pair from the rest positions (0 for point-triangle pairs
    and when mollification is off)."""
    out = np.zeros(len(pairs))
    if not MOLLIFY_EE or not len(pairs):
        return out
    P = np.asarray(pairs, dtype=np.int64).reshape(-1, 3)
    ee = P[:, 0] == 1
    if ee.any():
        Xr = np.asarray(scene.X, dtype=np.float64)
        ea, eb = scene.edges[P[ee, 1]], scene.edges[P[ee, 2]]
        u = Xr[ea[:, 1]] - Xr[ea[:, 0]]
        v = Xr[eb[:, 1]] - Xr[eb[:, 0]]
        out[ee] = MOLLIFIER_EPS * np.sum(u * u, axis=1) * np.sum(v * v, axis=1)
    return out


def _m_of_x(x, eps):
    X = x.reshape(4, 3)
    n = torch.linalg.cross(X[1] - X[0], X[3] - X[2])
    r = (n @ n) / eps
    return torch.where(r < 1.0, (2.0 - r) * r, torch.ones_like(r))


def mollifier(X4, eps, derivs=True):
    """m [n] (and grad m [n,12], Hessian of m [n,12,12]) of the edge-edge
    mollifier at stencil positions X4 [n,4,3]; rows with eps = 0 get m = 1."""
    n = X4.shape[0]
    m = np.ones(n)
    gm = np.zeros((n, 12))
    Hm = np.zeros((n, 12, 12))
    idx = np.flatnonzero(np.asarray(eps) > 0)
    if idx.size:
        xs = torch.from_numpy(np.ascontiguousarray(X4[idx].reshape(idx.size, 12))).double()
        es = torch.from_numpy(np.asarray(eps, dtype=np.float64)[idx])
        m[idx] = vmap(_m_of_x)(xs, es).numpy()
        if derivs:
            gm[idx] = vmap(grad(_m_of_x))(xs, es).numpy()
            Hm[idx] = vmap(hessian(_m_of_x))(xs, es).numpy()
    if derivs:
        return m, gm, Hm
    return m


def pair_energies(x, pairs, scene, inA, inAp, mu, s, sigma, dhat):
    """Per-pair energy phi_i at x (edge-edge pairs mollified), for the
    objective and the line search."""
    if not len(pairs):
        return np.zeros(0)
    d, _, nodes = pair_distances(x, pairs, scene)
    e, _, _ = phi_derivs(d, inA, inAp, mu, s, sigma, dhat)
    return e * mollifier(x[nodes], ee_eps(pairs, scene), derivs=False)


def normal_forces(x, pairs, scene, inA, inAp, mu, s, sigma, dhat):
    """Normal force magnitude -m phi'(d) of every pair at x (the lagged lambda
    of friction), with the distances' regions and the stencil nodes."""
    d, regions, nodes = pair_distances(x, pairs, scene)
    _, e1, _ = phi_derivs(d, inA, inAp, mu, s, sigma, dhat)
    m = mollifier(x[nodes], ee_eps(pairs, scene), derivs=False)
    return -m * e1, regions, nodes


def contact_terms(x, pairs, scene, inA, inAp, mu, s, sigma, dhat, project=True):
    """Per-pair energy [n], gradient [n,12], Hessian [n,12,12] (projected),
    stencil nodes [n,4] and distances [n]."""
    n = len(pairs)
    if n == 0:
        return (np.zeros(0), np.zeros((0, 12)), np.zeros((0, 12, 12)),
                np.zeros((0, 4), dtype=np.int64), np.zeros(0))
    nodes = stencil_nodes(pairs, scene)
    X4 = x[nodes]
    is_ee = np.asarray(pairs, dtype=np.int64).reshape(-1, 3)[:, 0] == 1
    regions = distance.classify(X4, is_ee)
    d, gd, Hd = distance.distance_derivatives(X4, regions)
    e, e1, e2 = phi_derivs(d, inA, inAp, mu, s, sigma, dhat)
    g = e1[:, None] * gd
    H = e2[:, None, None] * gd[:, :, None] * gd[:, None, :] + e1[:, None, None] * Hd
    m, gm, Hm = mollifier(X4, ee_eps(pairs, scene))
    H = (m[:, None, None] * H + e1[:, None, None] * (gd[:, :, None] * gm[:, None, :]
                                                     + gm[:, :, None] * gd[:, None, :])
         + e[:, None, None] * Hm)
    g = m[:, None] * g + e[:, None] * gm
    e = m * e
    if project:
        H = project_psd(H)
    return e, g, H, nodes, d


def _boxes(x, idx, dirv=None):
    """Axis-aligned boxes [n, 2, 3] of primitives idx [n, k] at x and, with dirv,
    at x + dirv (the box swept over the step)."""
    P = x[idx]
    lo, hi = P.min(axis=1), P.max(axis=1)
    if dirv is not None:
        Q = x[idx] + dirv[idx]
        lo, hi = np.minimum(lo, Q.min(axis=1)), np.maximum(hi, Q.max(axis=1))
    return lo, hi


def box_candidates(x, scene, r, dirv=None, chunk=2048):
    """Brute force over all PT pairs (surface vertex, surface triangle not
    containing it) and EE pairs (surface edges e < f sharing no vertex) whose
    boxes (swept along dirv if given) come within r on every axis:
    a.lo <= b.hi + r and b.lo <= a.hi + r. Sorted keys."""
    sv = scene.surf_verts.astype(np.int64)
    tris, edges = scene.tris.astype(np.int64), scene.edges.astype(np.int64)
    vlo, vhi = _boxes(x, sv[:, None], dirv)
    tlo, thi = _boxes(x, tris, dirv)
    elo, ehi = _boxes(x, edges, dirv)
    out = []

    def close(alo, ahi, blo, bhi):
        return np.all((alo[:, None, :] <= bhi[None, :, :] + r) & (blo[None, :, :] <= ahi[:, None, :] + r), axis=2)

    for s in range(0, len(sv), chunk):
        m = close(vlo[s:s + chunk], vhi[s:s + chunk], tlo, thi)
        iv, it = np.nonzero(m)
        v = sv[s + iv]
        keep = ~np.any(tris[it] == v[:, None], axis=1)
        out += list(zip([0] * int(keep.sum()), v[keep].tolist(), it[keep].tolist()))
    for s in range(0, len(edges), chunk):
        m = close(elo[s:s + chunk], ehi[s:s + chunk], elo, ehi)
        ie, jf = np.nonzero(m)
        e = s + ie
        keep = e < jf
        e, f = e[keep], jf[keep]
        share = np.any(edges[e][:, :, None] == edges[f][:, None, :], axis=(1, 2))
        out += [(1, int(a), int(b)) for a, b in zip(e[~share], f[~share])]
    out.sort()
    return out
