"""The two FP32 forms of H used by the FP32 + FP64-refinement solver, emulated
in NumPy FP32 arithmetic on the oracle's assembled H of a stiff system (a
3 x 3 piece of the chain net, 1 GPa links, border rings pinned):

- plain: every 3x3 block rounded to FP32, y_i = D_i v_i + sum_j B_ij v_j;
- difference: y_i = G_i v_i + sum_j B_ij (v_j - v_i), G_i = D_i + sum_j B_ij
  summed in FP64 and rounded once.

On a translation of one free link, H v = m/h^2 v (the stencil Hessians are
translation invariant). The difference form reproduces it to FP32 rounding;
the plain copy is off by more than the product itself (kappa eps_32 >> 1).
This pins the property the GPU solver's default operator form relies on."""
import numpy as np
import pytest

from oracle import system
from paper_2407_00046_b300 import scenes


@pytest.fixture(scope="module")
def stiff_net():
    sc = scenes.chain_net_shells(nx=3, nz=3, n_shells=0, link_theta=24, link_cross=2)
    m = system.make_model(sc)
    y = system.inertia_target(m, sc.X, sc.V0)
    H = system.hessian(m, sc.X, y, system.empty_pairs(), 0.0)
    n = sc.n_verts
    Hb = H.tobsr(blocksize=(3, 3))
    rows = np.repeat(np.arange(n), np.diff(Hb.indptr))
    cols = Hb.indices
    off = rows != cols
    D = np.zeros((n, 3, 3))
    D[rows[~off]] = Hb.data[~off]
    return sc, m, H, D, rows[off], cols[off], Hb.data[off]


def _plain(D, oi, oj, B, v):
    D32, B32, v32 = D.astype(np.float32), B.astype(np.float32), v.astype(np.float32)
    y = np.einsum("nab,nb->na", D32, v32).astype(np.float32)
    np.add.at(y, oi, np.einsum("nab,nb->na", B32, v32[oj]).astype(np.float32))
    return y.astype(np.float64)


def _difference(D, oi, oj, B, v):
    G = D.copy()
    np.add.at(G, oi, B)                               # FP64 row sums, one rounding below
    G32, B32, v32 = G.astype(np.float32), B.astype(np.float32), v.astype(np.float32)
    y = np.einsum("nab,nb->na", G32, v32).astype(np.float32)
    d = (v32[oj] - v32[oi]).astype(np.float32)
    np.add.at(y, oi, np.einsum("nab,nb->na", B32, d).astype(np.float32))
    return y.astype(np.float64)


def test_difference_form_is_h_in_exact_arithmetic(stiff_net):
    sc, m, H, D, oi, oj, B = stiff_net
    v = np.random.default_rng(0).normal(size=(sc.n_verts, 3))
    G = D.copy()
    np.add.at(G, oi, B)
    y = np.einsum("nab,nb->na", G, v)
    np.add.at(y, oi, np.einsum("nab,nb->na", B, v[oj] - v[oi]))
    ref = (H @ v.ravel()).reshape(-1, 3)
    assert np.abs(y - ref).max() <= 1e-9 * np.abs(ref).max()


def test_translations_are_exact_in_the_difference_form_only(stiff_net):
    sc, m, H, D, oi, oj, B = stiff_net
    free_bodies = [b for b in np.unique(sc.body) if not (sc.pinned[sc.body == b] == 1).any()]
    assert free_bodies
    idx = np.flatnonzero(sc.body == free_bodies[0])
    v = np.zeros((sc.n_verts, 3))
    v[idx, 0] = 1.0
    hv = (H @ v.ravel()).reshape(-1, 3)
    # H v is the mass term on the translated link
    assert np.allclose(hv[idx, 0], m.mass[idx] / m.h ** 2, rtol=1e-6)
    e_diff = np.linalg.norm(_difference(D, oi, oj, B, v) - hv) / np.linalg.norm(hv)
    e_plain = np.linalg.norm(_plain(D, oi, oj, B, v) - hv) / np.linalg.norm(hv)
    assert e_diff < 1e-6
    assert e_plain > 1.0
