"""Helpers shared by the GPU parity tests (test infrastructure)."""
import numpy as np
import scipy.sparse as sp

from oracle import bal as obal
from oracle import system


def blocks_to_csr(nv, D, rows, cols, vals):
    """Symmetric matrix from diagonal blocks D [nv,3,3] and lower blocks
    (rows, cols, vals [n,3,3]) with rows > cols."""
    r_all, c_all, v_all = [], [], []

    def add(bi, bj, B):
        if len(bi) == 0:
            return
        r = (3 * bi[:, None, None] + np.arange(3)[None, :, None]).repeat(3, axis=2)
        c = (3 * bj[:, None, None] + np.arange(3)[None, None, :]).repeat(3, axis=1)
        r_all.append(r.ravel())
        c_all.append(c.ravel())
        v_all.append(B.ravel())

    ar = np.arange(nv)
    add(ar, ar, D)
    add(rows, cols, vals)
    add(cols, rows, np.swapaxes(vals, 1, 2))
    n = 3 * nv
    return sp.coo_matrix((np.concatenate(v_all), (np.concatenate(r_all), np.concatenate(c_all))),
                         shape=(n, n)).tocsr()


def gpu_hessian(S, view):
    h = S.copy_hessian(view)
    nv = S.nv
    rp, col = S.static_pattern()
    rows = np.repeat(np.arange(nv), np.diff(rp))
    D = h["D"].cpu().numpy().reshape(nv, 3, 3)
    L = h["L"].cpu().numpy().reshape(-1, 3, 3)
    Cr = h["C_row"].cpu().numpy().astype(np.int64)
    Cc = h["C_col"].cpu().numpy().astype(np.int64)
    Cv = h["C_val"].cpu().numpy().reshape(-1, 3, 3)
    H = blocks_to_csr(nv, D, np.concatenate([rows, Cr]), np.concatenate([col, Cc]),
                      np.concatenate([L, Cv], axis=0))
    return H, h["Lambda"].cpu().numpy(), dict(D=D, L=L, rows=rows, cols=col, Cr=Cr, Cc=Cc, Cv=Cv)


def oracle_state(sc, x, sigma, ap=None):
    """Oracle model, y, pair set and assembled quantities at x for AL state
    (sigma, A' = ap dict key -> mu)."""
    m = system.make_model(sc)
    y = system.inertia_target(m, sc.X, sc.V0)
    keys, _ = obal.active_pairs(m, x)
    ps = obal.make_pairset(m, x, keys, ap or {}, sigma)
    return m, y, ps


def close_cubes(n=3, gap=4e-4, shift=0.013):
    from paper_2407_00046_b300 import scenes
    sc = scenes.two_cubes(n=n)
    sc.X[sc.body == 1, 1] -= 0.01 - gap
    sc.X[sc.body == 1, 0] += shift
    return sc
