"""Cubic continuous collision detection with a conservative time of impact,
FP64 (test infrastructure; Sec. 5.3, narrow phase).

A contact stencil moves along x(t) = x + t p, t in [0, 1]. Its four nodes are
coplanar where the triple product

    PT (p, t0, t1, t2):  f(t) = ((t1 - t0) x (t2 - t0)) . (p - t0)
    EE (a0, a1, b0, b1): f(t) = ((a1 - a0) x (b1 - b0)) . (b0 - a0)

vanishes; f is a cubic in t (each difference vector is linear in t). Steps in
the paper's order:

1. The first root t* of f in [-eps, 1 + eps] by a Newton-bisection root finder
   (the interval is split at the critical points of f, so each piece is
   monotone, and the earliest piece with a sign change is searched).
2. Deflation: f(t) = (t - t*)(A t^2 + B t + C) with A = a, B = b + A t*,
   C = c + B t*, whose roots in (t*, 1 + eps] are the later coplanar times.
3. Activation: at each coplanar time (time of coplanarity, TOC) in increasing
   order the unsigned distance d_TOC of the stencil is evaluated; the first
   with d_TOC < eps + dhat (eps = 1e-12) is the pair's time of impact. Reading:
   that threshold applies to a pair that starts outside the barrier's support
   (d(0) >= dhat); a pair already inside it (d(0) < dhat) is held off by the
   barrier itself, and activates only when it touches at a coplanar time
   (d_TOC < eps). Without this, two parallel edges closer than dhat -- always
   coplanar -- would give a zero step to every resting contact of flat faces.
4. Conservative TOI: with the previous coplanar time (or 0) t_prev, the
   reference frame t_ref = (t_prev + t_TOI) / 2 lies on the pre-crossing side;
   the returned time is multiplied by 0.9 until f there has the sign of
   f(t_ref) (and is non-zero). The triple product serves as the signed
   distance for every region (it is the plane distance times |n|).

Readings where the paper is silent: a stencil whose cubic vanishes
identically (all coefficients below 1e-14 L^3, L the stencil's extent plus
its motion) never crosses its plane and does not bound the step; roots are
polished to 1e-15 relative; at most 64 backtracking factors of 0.9 are taken.
The step bound of a line search is the minimum over the candidate pairs of
their conservative TOI scaled by the line search's margin eta (0.9): the paper
is silent on a margin, and without one a step ends at the touching time, where
the log barrier is still finite (distances of 1e-19 m were reached); 1 when no
pair activates.
"""
import numpy as np

from . import contact, distance

EPS = 1e-12
BACKTRACK = 0.9


def cubic_coefficients(X, P, is_ee):
    """Coefficients (c0, c1, c2, c3) of f(t) = c0 + c1 t + c2 t^2 + c3 t^3 for
    stencils X, P [n, 4, 3] (positions and displacements)."""
    if is_ee:
        u0, u1 = X[:, 1] - X[:, 0], P[:, 1] - P[:, 0]
        w0, w1 = X[:, 3] - X[:, 2], P[:, 3] - P[:, 2]
        v0, v1 = X[:, 2] - X[:, 0], P[:, 2] - P[:, 0]
    else:
        u0, u1 = X[:, 2] - X[:, 1], P[:, 2] - P[:, 1]
        w0, w1 = X[:, 3] - X[:, 1], P[:, 3] - P[:, 1]
        v0, v1 = X[:, 0] - X[:, 1], P[:, 0] - P[:, 1]
    n0 = np.cross(u0, w0)
    n1 = np.cross(u0, w1) + np.cross(u1, w0)
    n2 = np.cross(u1, w1)
    dot = lambda a, b: np.sum(a * b, axis=-1)  # noqa: E731
    return np.stack([dot(n0, v0), dot(n0, v1) + dot(n1, v0), dot(n1, v1) + dot(n2, v0),
                     dot(n2, v1)], axis=-1)


def _poly(c, t):
    return ((c[3] * t + c[2]) * t + c[1]) * t + c[0]


def _dpoly(c, t):
    return (3.0 * c[3] * t + 2.0 * c[2]) * t + c[1]


def _quadratic_roots(a, b, c):
    """Real roots of a t^2 + b t + c (a may be 0), stable form, ascending."""
    if a == 0.0:
        if b == 0.0:
            return []
        return [-c / b]
    disc = b * b - 4.0 * a * c
    if disc < 0.0:
        return []
    sq = np.sqrt(disc)
    q = -0.5 * (b + np.copysign(sq, b))
    r = [q / a] if q == 0.0 else [q / a, c / q]
    return sorted(r)


def _newton_bisect(c, lo, hi, flo):
    """Root of f in [lo, hi] with sign(f(lo)) = sign(flo) != sign(f(hi)):
    Newton steps kept inside the bracket, bisection otherwise."""
    t = 0.5 * (lo + hi)
    for _ in range(200):
        ft = _poly(c, t)
        if ft == 0.0:
            return t
        if (ft > 0) == (flo > 0):
            lo = t
        else:
            hi = t
        d = _dpoly(c, t)
        tn = t - ft / d if d != 0.0 else 0.5 * (lo + hi)
        if not (lo < tn < hi):
            tn = 0.5 * (lo + hi)
        if abs(tn - t) <= 1e-15 * max(1.0, abs(t)) or hi - lo <= 1e-16:
            return tn
        t = tn
    return t


def first_root(c, lo=-EPS, hi=1.0 + EPS):
    """Earliest root of the cubic c in [lo, hi] (None if f keeps one sign)."""
    crit = [t for t in _quadratic_roots(3.0 * c[3], 2.0 * c[2], c[1]) if lo < t < hi]
    knots = [lo] + crit + [hi]
    for a, b in zip(knots[:-1], knots[1:]):
        fa, fb = _poly(c, a), _poly(c, b)
        if fa == 0.0:
            return a
        if (fa > 0) != (fb > 0) or fb == 0.0:
            if fb == 0.0:
                return b
            return _newton_bisect(c, a, b, fa)
    return None


def coplanar_times(c, lo=-EPS, hi=1.0 + EPS):
    """Coplanar times in [lo, hi], ascending: the first root, then the roots of
    the deflated quadratic that lie after it."""
    t0 = first_root(c, lo, hi)
    if t0 is None:
        return []
    A = c[3]
    B = c[2] + A * t0
    C = c[1] + B * t0
    rest = [t for t in _quadratic_roots(A, B, C) if t0 < t <= hi]
    return [t0] + sorted(rest)


def pair_toi(X, P, is_ee, dhat, eta=1.0):
    """Conservative time of impact of one stencil (X, P [4, 3]) times eta; 1.0
    if it does not activate within [0, 1]."""
    c = cubic_coefficients(X[None], P[None], is_ee)[0]
    L = float(np.max(np.abs(X - X[0])) + np.max(np.abs(P - P[0])))
    if L == 0.0 or np.max(np.abs(c)) <= 1e-14 * (L * L * L):
        return 1.0
    times = coplanar_times(c)
    X0 = X[None]
    d0 = float(distance.distances(X0, distance.classify(X0, np.array([is_ee])))[0])
    thr = EPS + dhat if d0 >= dhat else EPS
    t_prev = 0.0
    for t in times:
        Xt = (X + t * P)[None]
        d = float(distance.distances(Xt, distance.classify(Xt, np.array([is_ee])))[0])
        if d < thr:
            t_ref = 0.5 * (max(t_prev, 0.0) + max(t, 0.0))
            f_ref = _poly(c, t_ref)
            tr = max(t, 0.0)
            for _ in range(64):
                ft = _poly(c, tr)
                if ft != 0.0 and (ft > 0) == (f_ref > 0):
                    break
                tr *= BACKTRACK
            return min(1.0, eta * tr)
        t_prev = t
    return 1.0


def step_bound(model, x, p, pairs, eta=0.9):
    """Minimum over the candidate pairs along x + t p of eta times their
    conservative TOI (1 for pairs that do not activate)."""
    if not pairs:
        return 1.0
    sc = model.scene
    nodes = contact.stencil_nodes(pairs, sc)
    X, P = x[nodes], p[nodes]
    is_ee = np.asarray(pairs, dtype=np.int64).reshape(-1, 3)[:, 0] == 1
    return float(min(pair_toi(X[i], P[i], bool(is_ee[i]), model.dhat, eta) for i in range(len(pairs))))
