"""Algorithm 1 (barrier-augmented Lagrangian) with exact linear solves: the
FP64 reference time step (test infrastructure).

One backward-Euler step (Sec. 3.1) minimises L_sigma by the primal-dual loop
of Algorithm 1 (Sec. 3.3) with the schedule of Sec. 3.4. Readings of the
paper used here (each one is recorded in the design notes):

* one loop iteration l = one inexact Newton step (assemble, solve, line
  search) followed by the dual update; the convergence test uses
  e = grad L at x^[l] and, when it passes, x^[l] is returned;
* "min d^[l+1]" in the A' rule is the minimum distance over A at the current
  iterate, compared with the value of the previous iteration (min of the
  empty set = +inf);
* A' rebuilds keep mu for pairs that stay in A'; dropped pairs lose it;
* s_i = max(-mu_i/sigma - dhat + d_i, 0) is evaluated at the start of an
  iteration and held fixed inside it; the dual update re-evaluates it at the
  new iterate before mu_i += sigma b(d_i, dhat + s_i);
* sigma update: sigma <- max(1.2 sigma, 100 sigma0) whenever min d < 1e-2 dhat,
  as printed (Alg. 1): a jump to 100 sigma0, then 1.2x growth per iteration
  until the closest pair is back above 1e-2 dhat; the capped reading
  min(1.2 sigma, 100 sigma0) is `sigma_literal_max = False`;
* sigma0 = -(sum grad b)^T grad E / ||sum grad b||^2 over A (the printed
  denominator is not squared, which is not dimensionally consistent), floored
  at mbar / (h^2 b''(dhat/2, dhat)); evaluated at x_0, or, when A(x_0) is empty,
  at the first iterate where A becomes non-empty;
* line search: alpha_0 = the largest t <= 1 along x + t p over which every pair
  keeps 10% of its current distance, found per pair by conservative
  advancement with Delta_i = max |p_a - p_b| over a node of each primitive as
  the bound on how fast the pair can close (an additive-CCD style time of
  impact in place of the paper's cubic CCD, Sec. 5.3); the candidate radius
  dhat + 2 max|p_v| / 0.9 contains every pair that can constrain alpha or
  enter A during the step; halve until no tet is
  inverted, the number of active pairs is within the memory cap (Sec. 5.2),
  and L_sigma does not increase by more than a rounding slack;
* friction (Sec. 4.1, chi > 0): lambda, the normal and the closest-point
  weights of every pair of A u A' are lagged at x^[l] after the A' rule and
  s_i are settled, held fixed through the gradient, the Hessian and the line
  search of that iteration, and refreshed at the next one; sigma0 and the
  dual update see no friction.
"""
import dataclasses
import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from . import barrier, ccd, contact, distance, elastic, friction
from .system import PairSet, energy_parts, gradient, hessian, inertia_target


@dataclasses.dataclass
class Params:
    newton_tol: float = 1e-4        # ||e^l|| / ||e^0|| (Alg. 1)
    newton_abs_tol: float = 0.0
    newton_max: int = 200
    ap_ratio: float = 1e-2          # A' threshold 1e-2 dhat (Alg. 1)
    sigma_growth: float = 1.2
    sigma_cap: float = 100.0
    sigma_literal_max: bool = True
    step_bound: float = 0.9
    ls_min_alpha: float = 1e-9      # App. B
    ls_slack: float = 1e-12
    contact_cap: int = 1 << 30      # Sec. 5.2 memory limit on |A|
    ca_max_iter: int = 64           # conservative-advancement iterations per pair
    freeze_al: bool = False         # hold sigma, A', mu fixed (adjoint checks)
    step_mode: str = "ca"           # "ca": conservative advancement; "ccd": cubic CCD (Sec. 5.3)
    al_mode: str = "bal"            # "bal": Algorithm 1; "plain": barrier with sigma = sigma0, A' empty
    broad_phase: str = "grid"       # line-search candidates: "grid" (radius rule) or "lbvh"
                                    # (boxes swept along the step within dhat)
    friction: float = 0.0           # chi (Sec. 4.1); 0 = frictionless
    eps_v: float = 0.0              # mollifier threshold (m/s); 0 = dhat (Table 1 caption)
    elastic_projection: str = "F"   # "F": 9x9 dP/dF (both paths); "stencil": 12x12 element block


def sigma_floor(model):
    b2 = float(barrier.d2b(np.array([model.dhat / 2]), model.dhat)[0])
    return float(np.mean(model.mass)) / (model.h ** 2 * b2)


def active_pairs(model, x):
    """A at x: pairs with d < dhat (sorted keys) and their distances."""
    cand = contact.candidate_pairs(x, model.scene, model.dhat)
    if not cand:
        return [], np.zeros(0)
    d, _, _ = contact.pair_distances(x, cand, model.scene)
    keep = d < model.dhat
    return [k for k, m in zip(cand, keep) if m], d[keep]


def initial_sigma(model, x, y, A_keys):
    floor = sigma_floor(model)
    if not A_keys:
        return floor
    n = len(A_keys)
    ps = PairSet(A_keys, np.ones(n, bool), np.zeros(n, bool), np.zeros(n), np.zeros(n))
    _, gE, gb = gradient(model, x, y, ps, 1.0, parts=True)
    nb2 = float(np.sum(gb * gb))
    if nb2 <= 0.0:
        return floor
    return max(-float(np.sum(gb * gE)) / nb2, floor)


def sigma_update(sigma, sigma0, dmin, prm: Params, dhat):
    """Alg. 1 line 16: when min d < 1e-2 dhat, sigma <- max(1.2 sigma, 100 sigma0)
    (the printed rule, `sigma_literal_max`) or min(1.2 sigma, 100 sigma0) (the
    capped reading); otherwise sigma is kept."""
    if not dmin < prm.ap_ratio * dhat:
        return sigma
    if prm.sigma_literal_max:
        return max(prm.sigma_growth * sigma, prm.sigma_cap * sigma0)
    return min(prm.sigma_growth * sigma, prm.sigma_cap * sigma0)


def augmentation_set(Ap, A_keys, A_d, dmin, dmin_prev, prm: Params, dhat):
    """Alg. 1 lines 3-6: A' = {} when min d > 1e-2 dhat; rebuilt from the pairs
    of A with d < 1e-2 dhat when min d fell below the previous iterate's or A'
    is empty (mu kept for pairs that stay, 0 for new ones); kept otherwise.
    Ap maps pair key -> mu; returns the new map."""
    thr = prm.ap_ratio * dhat
    if dmin > thr:
        return {}
    if dmin < dmin_prev or not Ap:
        return {k: Ap.get(k, 0.0) for k, dd in zip(A_keys, A_d) if dd < thr}
    return dict(Ap)


def dual_update(Ap, d_ap, sigma, dhat):
    """Alg. 1 lines 12-15 for every pair of A' (keys in sorted order, distances
    d_ap at the new iterate): s_i re-evaluated there (Sec. 3.2.2), then
    mu_i += sigma b(d_i, dhat + s_i)."""
    out = {}
    for k, dd in zip(sorted(Ap), d_ap):
        mu = Ap[k]
        s = max(-mu / sigma - dhat + dd, 0.0)
        out[k] = mu + sigma * float(barrier.b(np.array([dd]), dhat + s)[0])
    return out


def make_pairset(model, x, A_keys, Ap, sigma):
    keys = sorted(set(A_keys) | set(Ap))
    if not keys:
        return PairSet([], np.zeros(0, bool), np.zeros(0, bool), np.zeros(0), np.zeros(0))
    Aset = set(A_keys)
    inA = np.array([k in Aset for k in keys])
    inAp = np.array([k in Ap for k in keys])
    mu = np.array([Ap.get(k, 0.0) for k in keys])
    d, _, _ = contact.pair_distances(x, keys, model.scene)
    s = np.where(inAp, np.maximum(-mu / sigma - model.dhat + d, 0.0), 0.0)
    return PairSet(keys, inA, inAp, mu, s)


def displacement_bound(pairs, p, scene):
    """Delta_i = max over node a of the first primitive and node b of the second
    of |p_a - p_b|. Every point of the two convex hulls moves by a convex
    combination of node displacements, so the distance between the hulls can
    shrink by at most alpha * Delta_i along x + alpha p."""
    nodes = contact.stencil_nodes(pairs, scene)
    P = p[nodes]                                      # [n,4,3]
    is_pt = np.asarray(pairs, dtype=np.int64).reshape(-1, 3)[:, 0] == 0
    nrm = lambda a, b: np.sqrt(np.sum((P[:, a] - P[:, b]) ** 2, axis=1))  # noqa: E731
    pt = np.maximum(np.maximum(nrm(0, 1), nrm(0, 2)), nrm(0, 3))
    ee = np.maximum(np.maximum(nrm(0, 2), nrm(0, 3)), np.maximum(nrm(1, 2), nrm(1, 3)))
    return np.where(is_pt, pt, ee)


def step_bound(model, x, p, pairs, prm: Params):
    """Largest alpha <= 1 along x + t p over which every pair keeps at least
    (1 - step_bound) of its current distance d0, by conservative advancement:
    d can shrink by at most Delta per unit t (Delta = max |p_a - p_b|), so from t
    with distance d(t) it is safe to advance by (d(t) - (1 - eta) d0) / Delta.
    Iterate until the target distance is reached (the time of impact of the
    offset surface) or t = 1, at most ca_max_iter times per pair."""
    if not pairs:
        return 1.0
    sc = model.scene
    eta = prm.step_bound
    d0, _, _ = contact.pair_distances(x, pairs, sc)
    Dl = displacement_bound(pairs, p, sc)
    m = eta * d0 < Dl
    if not np.any(m):
        return 1.0
    keys = [k for k, f in zip(pairs, m) if f]
    d0, Dl = d0[m], Dl[m]
    goal = (1.0 - eta) * d0
    nodes = contact.stencil_nodes(keys, sc)
    X0, P0 = x[nodes], p[nodes]                         # [n,4,3]
    is_ee = np.asarray(keys, dtype=np.int64).reshape(-1, 3)[:, 0] == 1
    t = np.zeros(len(keys))
    active = np.ones(len(keys), dtype=bool)
    for _ in range(prm.ca_max_iter):
        idx = np.flatnonzero(active)
        if idx.size == 0:
            break
        X4 = X0[idx] + t[idx, None, None] * P0[idx]
        dk = distance.distances(X4, distance.classify(X4, is_ee[idx]))
        step = (dk - goal[idx]) / Dl[idx]
        done_toi = step <= 1e-6 * np.maximum(t[idx], 1e-3)
        newt = t[idx] + step
        reach = newt >= 1.0
        t[idx] = np.where(done_toi, t[idx], np.minimum(newt, 1.0))
        active[idx] = ~(done_toi | reach)
    return float(min(1.0, t.min()))


def friction_set(model, x, x_t, ps: PairSet, sigma, prm: Params):
    """Friction data of the pairs of ps lagged at x (None when chi = 0)."""
    if prm.friction <= 0.0 or not ps.keys:
        return None
    lam, regions, nodes = contact.normal_forces(x, ps.keys, model.scene, ps.inA, ps.inAp, ps.mu,
                                                ps.s, sigma, model.dhat)
    eps_v = prm.eps_v if prm.eps_v > 0.0 else model.dhat
    return friction.lag(x, x_t, nodes, regions, lam, prm.friction, eps_v * model.h)


def line_search(model, x, y, p, ps: PairSet, sigma, prm: Params, fric=None):
    sc = model.scene
    pnorm = np.sqrt(np.sum(p * p, axis=1))
    delta = float(pnorm[sc.surf_verts].max()) if sc.surf_verts.size else 0.0
    r = model.dhat + 2.0 * delta / prm.step_bound
    if prm.broad_phase == "lbvh":
        cand = contact.box_candidates(x, sc, model.dhat, p)
    else:
        cand = contact.candidate_pairs(x, sc, r)
    if prm.step_mode == "ccd":
        alpha = ccd.step_bound(model, x, p, cand, prm.step_bound)
    else:
        alpha = step_bound(model, x, p, cand, prm)
    parts_old = energy_parts(model, x, y, ps, sigma, fric)
    E_old = sum(parts_old)
    slack = prm.ls_slack * sum(abs(t) for t in parts_old)
    Ap_idx = [i for i, f in enumerate(ps.inAp) if f]
    Ap_keys = {ps.keys[i]: (ps.mu[i], ps.s[i]) for i in Ap_idx}
    trials = 0
    while alpha >= prm.ls_min_alpha:
        trials += 1
        xn = x + alpha * p
        F = elastic.deformation_gradient(xn, sc.tets, model.Dm_inv)
        if np.any(np.linalg.det(F) <= 0):
            alpha *= 0.5
            continue
        if cand:
            dn, _, _ = contact.pair_distances(xn, cand, sc)
            A_new = [k for k, dd in zip(cand, dn) if dd < model.dhat]
        else:
            A_new = []
        if len(A_new) > prm.contact_cap:
            alpha *= 0.5
            continue
        keys = sorted(set(A_new) | set(Ap_keys))
        Aset = set(A_new)
        psn = PairSet(keys, np.array([k in Aset for k in keys], dtype=bool),
                      np.array([k in Ap_keys for k in keys], dtype=bool),
                      np.array([Ap_keys.get(k, (0.0, 0.0))[0] for k in keys]),
                      np.array([Ap_keys.get(k, (0.0, 0.0))[1] for k in keys]))
        E_new = sum(energy_parts(model, xn, y, psn, sigma, fric))
        if E_new - E_old <= slack:
            return alpha, xn, dict(trials=trials, E_old=E_old, E_new=E_new,
                                   n_cand=len(cand))
        alpha *= 0.5
    return 0.0, x, dict(trials=trials, E_old=E_old, failed=True, n_cand=len(cand))


def solve(H, rhs):
    n = H.shape[0]
    if n <= 12000:
        c = sla.cho_factor(H.toarray(), lower=True)
        return sla.cho_solve(c, rhs)
    return spla.splu(H.tocsc()).solve(rhs)


def time_step(model, x_t, v_t, prm: Params = Params(), log=None, frozen=None):
    """One BAL time step from (x_t, v_t). Returns (x_{t+1}, v_{t+1}, info).
    frozen = (sigma, {A' key: mu}) holds the AL state fixed (no dual update, no
    sigma schedule, no A' rule): the map the adjoint differentiates."""
    dh = model.dhat
    y = inertia_target(model, x_t, v_t)
    x = np.array(x_t, dtype=np.float64, copy=True)
    A_keys, A_d = active_pairs(model, x)
    if frozen is not None:
        sigma0, Ap = frozen[0], dict(frozen[1])
    else:
        sigma0, Ap = initial_sigma(model, x, y, A_keys), {}
    # the formula needs A != empty: when the step starts contact-free, sigma0 is
    # taken at the first iterate where A becomes non-empty
    sigma0_pending = frozen is None and not A_keys
    sigma = sigma0
    dmin_prev = math.inf
    info = dict(sigma0=sigma0, iters=0, converged=False, ls_failed=False, log=[])
    e0 = None
    for l in range(prm.newton_max):
        if l > 0:
            A_keys, A_d = active_pairs(model, x)
        dmin = float(A_d.min()) if A_d.size else math.inf
        if sigma0_pending and A_keys:
            sigma0 = initial_sigma(model, x, y, A_keys)
            sigma = sigma0
            sigma0_pending = False
            info["sigma0"] = sigma0
        plain = prm.al_mode == "plain"   # ablation: the plain inexact Newton method
        if l > 0 and frozen is None and not plain:
            # dual update of the previous iteration, evaluated at x^[l]
            if Ap:
                d_ap, _, _ = contact.pair_distances(x, sorted(Ap), model.scene)
                Ap = dual_update(Ap, d_ap, sigma, dh)
            sigma = sigma_update(sigma, sigma0, dmin, prm, dh)
        # augmentation set rule (Alg. 1 lines 3-6)
        if plain:
            Ap = {}
        elif frozen is None:
            Ap = augmentation_set(Ap, A_keys, A_d, dmin, dmin_prev, prm, dh)
        dmin_prev = dmin
        ps = make_pairset(model, x, A_keys, Ap, sigma)
        fs = friction_set(model, x, x_t, ps, sigma, prm)
        e = gradient(model, x, y, ps, sigma, fric=fs)
        en = float(np.linalg.norm(e))
        rec = dict(l=l, nA=len(A_keys), nAp=len(Ap), sigma=sigma, dmin=dmin, enorm=en)
        info["log"].append(rec)
        if e0 is None:
            e0 = en
        if en <= prm.newton_abs_tol or (l > 0 and en <= prm.newton_tol * e0):
            info["converged"] = True
            break
        H = hessian(model, x, y, ps, sigma, fric=fs, elastic_projection=prm.elastic_projection)
        p = solve(H, -e.ravel()).reshape(-1, 3)
        alpha, xn, lsi = line_search(model, x, y, p, ps, sigma, prm, fs)
        rec["alpha"] = alpha
        rec["ls_trials"] = lsi["trials"]
        info["iters"] = l + 1
        if lsi.get("failed"):
            info["ls_failed"] = True
            break
        x = xn
    info["sigma"] = sigma
    info["Ap"] = dict(Ap)
    v = (x - x_t) / model.h
    if log is not None:
        log.append(info)
    return x, v, info
