"""Fully-implicit friction (Sec. 4.1), FP64 (test infrastructure).

Per contact pair j (a PT or EE stencil of A u A') the dissipative potential of
Sec. 4.1 is

    D_j(x) = chi lambda_j f(|w_j|),   w_j = P_j Gamma_j (x - x_t),

with three quantities taken at the lag point x^[l] (the current Newton
iterate) and held fixed while D is differentiated and during the line search;
they are refreshed at every inexact Newton iteration (the per-iteration update
of Sec. 4.1):

  beta_j    signed barycentric weights of the two closest points, so that
            Gamma_j x = sum_k beta_jk x_k (Gamma_j = [beta_j0 I ... beta_j3 I])
            is the vector from the closest point of the second primitive to
            that of the first; |Gamma_j x^[l]| = d_j;
  n_j       the contact normal Gamma_j x^[l]; P_j = I - n_j n_j^T / (n_j . n_j)
            removes the normal part, so w_j = h u_j with u_j the tangent
            relative velocity of Sec. 4.1 (v_r = Gamma_j (x - x_t) / h);
  lambda_j  the magnitude of the pair's normal contact force,
            -d phi_j / dd at x^[l] with phi_j the pair's barrier + AL energy
            (Sec. 3.3), which is >= 0.

Mollifier (readings): f(y) = y^2 / (eps h) - y^3 / (3 eps^2 h^2) for
y < eps h, the printed form, continued by f(y) = y - eps h / 3 for y >= eps h
(the printed cubic covers only the static zone; the continuation is C^2 and
makes the sliding force exactly chi lambda, Coulomb's law). eps = eps_v, which
the paper sets numerically equal to dhat (Table 1 caption).

Derivatives (w is linear in x, so only f and |.| are differentiated):
    grad D_j = chi lambda_j a(y) Gamma^T w,              a = f'(y) / y
    Hess D_j = chi lambda_j Gamma^T (a P + c w w^T) Gamma, c = (f''(y) - a) / y^2
with a = 2/(eps h) - y/(eps h)^2, c y = -1/(eps h)^2 in the static zone
(finite at y = 0, where the c term vanishes) and a = 1/y, c = -1/y^3 beyond.
Both a and a + c y^2 = f'' are >= 0, so the friction Hessian is PSD without
projection.
"""
import dataclasses

import numpy as np

from . import distance


@dataclasses.dataclass
class FrictionSet:
    """Lagged friction data of the pairs with lambda > 0."""
    nodes: np.ndarray    # [n,4] stencil vertex ids
    beta: np.ndarray     # [n,4]
    normal: np.ndarray   # [n,3] n_j (not normalised)
    lam: np.ndarray      # [n]
    chi: float
    eps_h: float         # eps_v * h
    x_t: np.ndarray      # [N_v,3] start of the time step


def mollifier(y, eps_h):
    """f, f', f'' of the mollified friction magnitude (vectorised)."""
    y = np.asarray(y, dtype=np.float64)
    s = y < eps_h
    f = np.where(s, y * y / eps_h - y ** 3 / (3.0 * eps_h ** 2), y - eps_h / 3.0)
    f1 = np.where(s, 2.0 * y / eps_h - y * y / eps_h ** 2, 1.0)
    f2 = np.where(s, 2.0 / eps_h - 2.0 * y / eps_h ** 2, 0.0)
    return f, f1, f2


def _solve2(a11, a12, a22, r1, r2):
    """Batched 2x2 symmetric solve by numpy.linalg.solve."""
    A = np.stack([np.stack([a11, a12], -1), np.stack([a12, a22], -1)], -2)
    return np.linalg.solve(A, np.stack([r1, r2], -1)[..., None])[..., 0]


def closest_weights(X4, regions):
    """beta [n,4] of the closest points of each stencil, by region:
    PP (i, j): beta_i = 1, beta_j = -1;
    PE (p, a, b): t = (x_p - x_a).(x_b - x_a) / |x_b - x_a|^2,
                  beta_p = 1, beta_a = -(1 - t), beta_b = -t;
    PT: (b1, b2) minimising |p - t0 - b1 (t1 - t0) - b2 (t2 - t0)|
        (normal equations), beta = (1, -(1 - b1 - b2), -b1, -b2);
    EE: (s, t) minimising |a0 + s (a1 - a0) - b0 - t (b1 - b0)|
        (normal equations), beta = (1 - s, s, -(1 - t), -t).
    Signs are fixed so that the first primitive's weights are >= 0 (a PE
    region of an EE pair whose point is on the second edge is negated)."""
    X4 = np.asarray(X4, dtype=np.float64)
    n = X4.shape[0]
    beta = np.zeros((n, 4))
    for i, (kind, loc) in enumerate(regions):
        X = X4[i]
        if kind == distance.PP:
            beta[i, loc[0]], beta[i, loc[1]] = 1.0, -1.0
        elif kind == distance.PE:
            p, a, b = X[loc[0]], X[loc[1]], X[loc[2]]
            t = np.dot(p - a, b - a) / np.dot(b - a, b - a)
            beta[i, loc[0]], beta[i, loc[1]], beta[i, loc[2]] = 1.0, -(1.0 - t), -t
        elif kind == distance.PT:
            e1, e2, r = X[2] - X[1], X[3] - X[1], X[0] - X[1]
            b1, b2 = _solve2(np.dot(e1, e1), np.dot(e1, e2), np.dot(e2, e2),
                             np.dot(e1, r), np.dot(e2, r))
            beta[i] = (1.0, -(1.0 - b1 - b2), -b1, -b2)
        else:
            u, v, w = X[1] - X[0], X[3] - X[2], X[0] - X[2]
            s, t = _solve2(np.dot(u, u), -np.dot(u, v), np.dot(v, v), -np.dot(u, w), np.dot(v, w))
            beta[i] = (1.0 - s, s, -(1.0 - t), -t)
        if beta[i, 0] + beta[i, 1] < 0.0:    # an EE region led by edge b's point: first minus second
            beta[i] = -beta[i]
    return beta


def lag(x, x_t, nodes, regions, lam, chi, eps_h):
    """FrictionSet of the pairs with lambda > 0, lagged at x."""
    keep = np.asarray(lam) > 0
    nodes = np.asarray(nodes)[keep]
    regions = [r for r, k in zip(regions, keep) if k]
    X4 = x[nodes]
    beta = closest_weights(X4, regions)
    normal = np.einsum("nk,nkc->nc", beta, X4)
    return FrictionSet(nodes=nodes, beta=beta, normal=normal, lam=np.asarray(lam)[keep],
                       chi=float(chi), eps_h=float(eps_h), x_t=x_t)


def _tangent(fs: FrictionSet, x):
    """w [n,3] and the projector P [n,3,3]."""
    nn = fs.normal / np.linalg.norm(fs.normal, axis=1)[:, None]
    P = np.eye(3)[None] - nn[:, :, None] * nn[:, None, :]
    u = np.einsum("nk,nkc->nc", fs.beta, x[fs.nodes] - fs.x_t[fs.nodes])
    return np.einsum("nij,nj->ni", P, u), P


def energy(fs: FrictionSet, x):
    """sum_j D_j(x)."""
    if fs is None or fs.nodes.shape[0] == 0:
        return 0.0
    w, _ = _tangent(fs, x)
    f, _, _ = mollifier(np.linalg.norm(w, axis=1), fs.eps_h)
    return float(np.sum(fs.chi * fs.lam * f))


def terms(fs: FrictionSet, x, hessian=True):
    """Per-pair energy [n], gradient [n,12], Hessian [n,12,12] (or None)."""
    n = fs.nodes.shape[0]
    w, P = _tangent(fs, x)
    y = np.linalg.norm(w, axis=1)
    f, f1, f2 = mollifier(y, fs.eps_h)
    s = y < fs.eps_h
    eh = fs.eps_h
    a = np.where(s, 2.0 / eh - y / eh ** 2, 1.0 / np.where(s, 1.0, y))
    k = fs.chi * fs.lam
    G = np.einsum("nk,nc->nkc", fs.beta, w).reshape(n, 12)     # Gamma^T w
    g = (k * a)[:, None] * G
    if not hessian:
        return k * f, g, None
    # c w w^T: -(w w^T) / (eh^2 y) in the static zone (0 at y = 0), -(w w^T) / y^3 beyond
    ysafe = np.where(y > 0, y, 1.0)
    cy = np.where(s, -1.0 / eh ** 2 / ysafe, -1.0 / ysafe ** 3)
    cy = np.where(y > 0, cy, 0.0)
    M = a[:, None, None] * P + cy[:, None, None] * w[:, :, None] * w[:, None, :]
    H = np.einsum("nk,nl,nij->nkilj", fs.beta, fs.beta, M).reshape(n, 12, 12)
    return k * f, g, k[:, None, None] * H
