"""Unsigned distances of contact stencils with region classification, FP64
(test infrastructure).

A contact stencil is a point-triangle (PT) pair, nodes (p, t0, t1, t2), or an
edge-edge (EE) pair, nodes (a0, a1, b0, b1) (Sec. 5.3: "VF / EE ... or their
degenerate cases"). The barrier of Sec. 3.3 is written in the distance d
itself, so d is the unsigned Euclidean distance between the two primitives.
The closest-point problem is classified into a region, and in each region d^2
has a plain closed form in the active nodes only:

    PP  |p - q|^2
    PE  |(p - a) x (b - a)|^2 / |b - a|^2
    PT  ((p - t0) . n)^2 / |n|^2,     n = (t1 - t0) x (t2 - t0)
    EE  ((a0 - b0) . n)^2 / |n|^2,    n = (a1 - a0) x (b1 - b0)

Classification (same decision rule on every side, ties go to the
lower-dimensional region):
  PT: barycentric coordinates of the projection of p; strictly inside -> PT;
      otherwise the nearest of the three edges (t0t1, t1t2, t2t0, first wins
      on ties), each edge being PE if its clamped parameter is in (0, 1),
      else PP with the nearer end.
  EE: with n = u x v computed as a cross product, if |n|^2 > 1e-12 |u|^2 |v|^2
      (edges not within ~1e-6 rad of parallel; the threshold sits far above the
      FP64 rounding floor of the line-line parameters) and the line-line
      parameters are both in (0, 1) -> EE; otherwise the nearest of the four point-segment cases
      (a0 vs b, a1 vs b, b0 vs a, b1 vs a; first wins on ties).

Gradients and Hessians of d = sqrt(d^2) are taken by automatic
differentiation (torch.func, FP64) of the region formula, which is an
independent derivation from the hand-written ones in the CUDA kernels.
"""
import numpy as np
import torch
from torch.func import grad, hessian, vmap

# region kinds
PP, PE, PT, EE = 0, 1, 2, 3
PARALLEL_EPS = 1e-12




def _dot(a, b):
    return a[..., 0] * b[..., 0] + a[..., 1] * b[..., 1] + a[..., 2] * b[..., 2]


def _crossv(a, b):
    return np.stack([a[..., 1] * b[..., 2] - a[..., 2] * b[..., 1],
                     a[..., 2] * b[..., 0] - a[..., 0] * b[..., 2],
                     a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]], axis=-1)


def _seg_candidates(p, a, b):
    """Point-segment squared distance (closest point), kind and which end for PP.
    Returns d2 [n], kind [n] (PP or PE), end [n] (0 = a, 1 = b; PP only)."""
    ab = b - a
    L2 = _dot(ab, ab)
    with np.errstate(divide="ignore", invalid="ignore"):
        u = np.where(L2 > 0, _dot(p - a, ab) / np.where(L2 > 0, L2, 1.0), 0.0)
    c = a + u[:, None] * ab
    d2 = _dot(p - c, p - c)
    da, db = _dot(p - a, p - a), _dot(p - b, p - b)
    kind = np.where((u <= 0) | (u >= 1), PP, PE)
    end = np.where(u >= 1, 1, 0)
    d2 = np.where(u <= 0, da, np.where(u >= 1, db, d2))
    return d2, kind, end


def _pick(cands):
    """cands: list of (d2, kind, end, p, a, b) for k = 0.. in order; the first
    strictly smaller squared distance wins. Returns kind, loc tuples."""
    best = cands[0][0].copy()
    arg = np.zeros(best.shape, dtype=np.int64)
    for k in range(1, len(cands)):
        better = cands[k][0] < best
        best = np.where(better, cands[k][0], best)
        arg = np.where(better, k, arg)
    out = []
    for i in range(best.shape[0]):
        d2, kind, end, ip, ia, ib = cands[arg[i]]
        if kind[i] == PE:
            out.append((PE, (ip, ia, ib)))
        else:
            out.append((PP, (ip, ib if end[i] else ia)))
    return out


def classify_pt_batch(X4):
    p, t0, t1, t2 = X4[:, 0], X4[:, 1], X4[:, 2], X4[:, 3]
    e1, e2, r = t1 - t0, t2 - t0, p - t0
    a11, a12, a22 = _dot(e1, e1), _dot(e1, e2), _dot(e2, e2)
    b1, b2 = _dot(e1, r), _dot(e2, r)
    det = a11 * a22 - a12 * a12
    sdet = np.where(det > 0, det, 1.0)
    be1 = (a22 * b1 - a12 * b2) / sdet
    be2 = (a11 * b2 - a12 * b1) / sdet
    be0 = 1.0 - be1 - be2
    inside = (det > 0) & (be0 > 0) & (be1 > 0) & (be2 > 0)
    nodes = (p, t0, t1, t2)
    cands = []
    for (ia, ib) in ((1, 2), (2, 3), (3, 1)):
        d2, kind, end = _seg_candidates(p, nodes[ia], nodes[ib])
        cands.append((d2, kind, end, 0, ia, ib))
    edge = _pick(cands)
    return [(PT, (0, 1, 2, 3)) if inside[i] else edge[i] for i in range(len(edge))]


def classify_ee_batch(X4):
    a0, a1, b0, b1 = X4[:, 0], X4[:, 1], X4[:, 2], X4[:, 3]
    u, v, w = a1 - a0, b1 - b0, a0 - b0
    A, B, C, D, Ev = _dot(u, u), _dot(u, v), _dot(v, v), _dot(u, w), _dot(v, w)
    n = _crossv(u, v)
    den = _dot(n, n)
    nonpar = den > PARALLEL_EPS * A * C
    sden = np.where(nonpar, den, 1.0)
    s = (B * Ev - C * D) / sden
    t = (A * Ev - B * D) / sden
    interior = nonpar & (s > 0) & (s < 1) & (t > 0) & (t < 1)
    nodes = (a0, a1, b0, b1)
    cands = []
    for (ip, ia, ib) in ((0, 2, 3), (1, 2, 3), (2, 0, 1), (3, 0, 1)):
        d2, kind, end = _seg_candidates(nodes[ip], nodes[ia], nodes[ib])
        cands.append((d2, kind, end, ip, ia, ib))
    edge = _pick(cands)
    return [(EE, (0, 1, 2, 3)) if interior[i] else edge[i] for i in range(len(edge))]


def classify_pt(p, t0, t1, t2):
    """Returns (kind, node indices into (p, t0, t1, t2))."""
    return classify_pt_batch(np.stack([p, t0, t1, t2])[None])[0]


def classify_ee(a0, a1, b0, b1):
    """Returns (kind, node indices into (a0, a1, b0, b1))."""
    return classify_ee_batch(np.stack([a0, a1, b0, b1])[None])[0]


# ---- region formulas on a 12-vector (4 nodes x 3), torch FP64 ----------------
def _d2_pp(x, i, j):
    X = x.reshape(4, 3)
    r = X[i] - X[j]
    return r @ r


def _d2_pe(x, ip, ia, ib):
    X = x.reshape(4, 3)
    e = X[ib] - X[ia]
    c = torch.linalg.cross(X[ip] - X[ia], e)
    return (c @ c) / (e @ e)


def _d2_plane(x, i0, i1, i2, i3, kind):
    X = x.reshape(4, 3)
    if kind == PT:   # point X[i0], triangle X[i1], X[i2], X[i3]
        n = torch.linalg.cross(X[i2] - X[i1], X[i3] - X[i1])
        r = X[i0] - X[i1]
    else:            # edges X[i0]X[i1], X[i2]X[i3]
        n = torch.linalg.cross(X[i1] - X[i0], X[i3] - X[i2])
        r = X[i0] - X[i2]
    u = r @ n
    return u * u / (n @ n)


def d2_fn(kind, loc):
    if kind == PP:
        return lambda x: _d2_pp(x, *loc)
    if kind == PE:
        return lambda x: _d2_pe(x, *loc)
    return lambda x: _d2_plane(x, *loc, kind)


def distance_derivatives(X4, regions):
    """X4 [n,4,3] stencil node positions, regions list of (kind, loc).
    Returns d [n], grad d [n,12], Hessian of d [n,12,12] (FP64)."""
    n = len(regions)
    d = np.zeros(n)
    g = np.zeros((n, 12))
    H = np.zeros((n, 12, 12))
    groups = {}
    for i, r in enumerate(regions):
        groups.setdefault(r, []).append(i)
    for (kind, loc), idx in groups.items():
        f2 = d2_fn(kind, loc)
        f = lambda x, f2=f2: torch.sqrt(f2(x))  # noqa: E731
        xs = torch.from_numpy(np.ascontiguousarray(X4[idx].reshape(len(idx), 12))).double()
        d[idx] = vmap(f)(xs).numpy()
        g[idx] = vmap(grad(f))(xs).numpy()
        H[idx] = vmap(hessian(f))(xs).numpy()
    return d, g, H


def distances(X4, regions):
    """d only (no derivatives), FP64 numpy, for the line search."""
    out = np.zeros(len(regions))
    groups = {}
    for i, r in enumerate(regions):
        groups.setdefault(r, []).append(i)
    for (kind, loc), idx in groups.items():
        X = X4[idx]
        if kind == PP:
            r = X[:, loc[0]] - X[:, loc[1]]
            out[idx] = np.sqrt(_dot(r, r))
        elif kind == PE:
            e = X[:, loc[2]] - X[:, loc[1]]
            c = _crossv(X[:, loc[0]] - X[:, loc[1]], e)
            out[idx] = np.sqrt(_dot(c, c) / _dot(e, e))
        elif kind == PT:
            nrm = _crossv(X[:, loc[2]] - X[:, loc[1]], X[:, loc[3]] - X[:, loc[1]])
            out[idx] = np.abs(_dot(X[:, loc[0]] - X[:, loc[1]], nrm)) / np.sqrt(_dot(nrm, nrm))
        else:
            nrm = _crossv(X[:, loc[1]] - X[:, loc[0]], X[:, loc[3]] - X[:, loc[2]])
            out[idx] = np.abs(_dot(X[:, loc[0]] - X[:, loc[2]], nrm)) / np.sqrt(_dot(nrm, nrm))
    return out


def classify(X4, is_ee):
    X4 = np.asarray(X4, dtype=np.float64)
    is_ee = np.asarray(is_ee, dtype=bool)
    out = [None] * X4.shape[0]
    for flag, fn in ((False, classify_pt_batch), (True, classify_ee_batch)):
        idx = np.flatnonzero(is_ee == flag)
        if idx.size:
            for i, r in zip(idx, fn(X4[idx])):
                out[i] = r
    return out
