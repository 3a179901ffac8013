"""Parity at full workload sizes (663,552-tet cube stack, 1.77M-tet chain net,
1.05M-tet stack of 64 cubes in contact): sampled vertex rows of the assembled
Hessian and of the gradient against the oracle evaluated on the incident
stencils only (tets, and contact pairs where the bodies touch), plus
properties that hold at any size (SpMV symmetry, PCG residual)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import elastic  # noqa: E402
from paper_2407_00046_b300 import bal, scenes  # noqa: E402

DEV = "cuda"


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _oracle_rows(sc, x, verts, mass, project=True):
    """Blocks H[v, u] (3x3) and gradients g[v] from the elastic stencils of the
    tets incident to each sampled vertex plus the mass term (no contact)."""
    Dm_inv, vol = elastic.rest_data(sc.X, sc.tets)
    mu, lam = elastic.lame(sc.E, sc.nu)
    h = sc.h
    rows, grads = {}, {}
    for v in verts:
        tt = np.flatnonzero(np.any(sc.tets == v, axis=1))
        _, g, H = elastic.element_terms(x, sc.tets[tt], Dm_inv[tt], vol[tt], mu[tt], lam[tt], project)
        blocks = {v: np.eye(3) * mass[v] / h ** 2}
        gv = np.zeros(3)
        for k, t in enumerate(tt):
            a = int(np.flatnonzero(sc.tets[t] == v)[0])
            gv += g[k, 3 * a:3 * a + 3]
            for b in range(4):
                u = int(sc.tets[t, b])
                blocks[u] = blocks.get(u, np.zeros((3, 3))) + H[k, 3 * a:3 * a + 3, 3 * b:3 * b + 3]
        rows[v], grads[v] = blocks, gv
    return rows, grads


def _gpu_rows(S, view, verts):
    h = S.copy_hessian(view)
    nv = S.nv
    rp, col = S.static_pattern()
    D = h["D"].cpu().numpy().reshape(nv, 3, 3)
    L = h["L"].cpu().numpy().reshape(-1, 3, 3)
    out = {}
    for v in verts:
        blocks = {v: D[v]}
        for s in range(rp[v], rp[v + 1]):            # row v: blocks (v, col)
            blocks[int(col[s])] = L[s]
        for s in np.flatnonzero(col == v):            # column v: transposes of (row, v)
            r = int(np.searchsorted(rp, s, side="right") - 1)
            blocks[r] = L[s].T
        out[v] = blocks
    return out


@pytest.mark.parametrize("name", ["cube_stack", "chain_net_shells"])
def test_sampled_rows_at_full_size(name):
    sc = scenes.scene_by_name(name)
    rng = np.random.default_rng(9)
    S = bal.Scene(sc, bal.default_params(), pair_capacity=1 << 22)
    mass = S.mass()
    # a deformed, contact-free iterate: small random displacement of free vertices
    x = sc.X + 2e-5 * rng.normal(size=sc.X.shape) * (sc.pinned == 0)[:, None]
    S.step_begin(T(sc.X), T(sc.V0))
    g = torch.empty(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    view = S.assemble_hessian(T(x), g)
    assert view["nnz_C"] == 0
    free = np.flatnonzero(sc.pinned == 0)
    verts = [int(v) for v in rng.choice(free, 24, replace=False)]
    ro, go = _oracle_rows(sc, x, verts, mass)
    rg = _gpu_rows(S, view, verts)
    y = sc.X + sc.h * sc.V0 + sc.h ** 2 * sc.gravity[None, :]
    gg = g.cpu().numpy().reshape(-1, 3)
    for v in verts:
        scale = max(np.abs(B).max() for B in ro[v].values())
        for u, B in ro[v].items():
            if sc.pinned[u]:
                continue
            assert np.abs(rg[v][u] - B).max() <= 1e-10 * scale, (v, u)
        ref = go[v] + mass[v] * (x[v] - y[v]) / sc.h ** 2
        assert np.abs(gg[v] - ref).max() <= 1e-10 * max(np.abs(ref).max(), 1e-30)
    # properties at full size: symmetric SpMV, PCG residual
    u1 = torch.randn(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    u2 = torch.randn_like(u1)
    h1, h2 = torch.empty_like(u1), torch.empty_like(u1)
    S.spmv(u1, h1)
    S.spmv(u2, h2)
    a, b = float(u2 @ h1), float(u1 @ h2)
    assert abs(a - b) <= 1e-11 * max(abs(a), abs(b))
    sol = torch.zeros_like(u1)
    info = S.pcg_solve(-g, sol, 1e-6, 1000)
    assert info["iters"] > 0 and np.isfinite(info["rel_residual"])


def test_df64_solve_at_full_size():
    """The benchmark's solver in its launch configuration (double-float PCG,
    sliced-ELL SpMV, 1.77M-tet net, first Newton system of a step, relative
    tolerance 1e-6, stagnation window 5000): every sampled residual row,
    b_v - sum_u H_vu x_u with the oracle's rows of H and of b = -grad, stays
    below the tolerance times ||b||, as a 2-norm bound on the whole residual
    requires of each of its rows. Allowance for the two assemblies' rounding:
    100 FP64 ulps of each row's sum of |H_vu x_u| (stiff 1 GPa rows sum terms
    ~1e6 times larger than ||b||)."""
    sc = scenes.scene_by_name("chain_net_shells")
    rng = np.random.default_rng(10)
    S = bal.Scene(sc, bal.default_params(precision=bal.PREC_DF64, pcg_stall_window=5000,
                                         pcg_max_iter=30000), pair_capacity=1 << 22)
    mass = S.mass()
    x = sc.X.copy()
    S.step_begin(T(sc.X), T(sc.V0))
    g = torch.empty(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    S.assemble_hessian(T(x), g)
    sol = torch.zeros_like(g)
    tol = 1e-6
    info = S.pcg_solve(-g, sol, tol, 30000)
    assert info["converged"] == 1 and info["precision_used"] == bal.PREC_DF64
    free = np.flatnonzero(sc.pinned == 0)
    verts = [int(v) for v in rng.choice(free, 24, replace=False)]
    ro, go = _oracle_rows(sc, x, verts, mass)
    y = sc.X + sc.h * sc.V0 + sc.h ** 2 * sc.gravity[None, :]
    xs = sol.cpu().numpy().reshape(-1, 3)
    bnorm = float(torch.linalg.norm(g))
    for v in verts:
        b_v = -(go[v] + mass[v] * (x[v] - y[v]) / sc.h ** 2)
        terms = [B @ xs[u] for u, B in ro[v].items() if not sc.pinned[u]]
        r_v = b_v - sum(terms)
        scale = sum(np.abs(B) @ np.abs(xs[u]) for u, B in ro[v].items() if not sc.pinned[u])
        bound = 1.01 * tol * bnorm + 100 * np.finfo(np.float64).eps * np.linalg.norm(scale)
        assert np.linalg.norm(r_v) <= bound, (v, np.linalg.norm(r_v), bound)


def _gpu_rows_with_contact(S, view, verts):
    """GPU rows of D + L + L^T + C + C^T at the sampled vertices."""
    out = _gpu_rows(S, view, verts)
    h = S.copy_hessian(view)
    Cr = h["C_row"].cpu().numpy().astype(np.int64)
    Cc = h["C_col"].cpu().numpy().astype(np.int64)
    Cv = h["C_val"].cpu().numpy().reshape(-1, 3, 3)
    for v in verts:
        for k in np.flatnonzero(Cr == v):
            out[v][int(Cc[k])] = out[v].get(int(Cc[k]), np.zeros((3, 3))) + Cv[k]
        for k in np.flatnonzero(Cc == v):
            out[v][int(Cr[k])] = out[v].get(int(Cr[k]), np.zeros((3, 3))) + Cv[k].T
    return out


def test_sampled_rows_in_contact_at_full_size():
    """The 1.05M-tet stack of 64 cubes (E log-uniform in [1e5, 1e9]) with the
    cubes unrotated and 0.3 mm apart, perturbed by 20 um: every stacked pair of
    faces is in contact (about 1e5 active point-triangle and edge-edge pairs,
    many of them near-parallel edges inside the mollified zone). Sampled rows
    of the assembled Hessian (elastic, contact, mass) and of the gradient
    against the oracle's stencils incident to each sampled vertex."""
    from oracle import bal as obal
    from oracle import contact, system
    sc = scenes.cube_columns(max_rot_deg=0.0, gap=3e-4)
    rng = np.random.default_rng(12)
    x = sc.X + 2e-5 * rng.normal(size=sc.X.shape) * (sc.pinned == 0)[:, None]
    S = bal.Scene(sc, bal.default_params(), pair_capacity=1 << 22)
    mass = S.mass()
    S.step_begin(T(sc.X), T(sc.V0))                   # sigma0 from the contact at the 0.3 mm gaps
    al = S.get_al_state()
    sigma = al["sigma"]
    g = torch.empty(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    view = S.assemble_hessian(T(x), g)
    assert view["nnz_C"] > 5e4
    # sampled vertices: on the contact faces and anywhere else
    cand = contact.candidate_pairs(x, sc, sc.dhat)
    nodes = contact.stencil_nodes(cand, sc)
    d, _, _ = contact.pair_distances(x, cand, sc)
    active = d < sc.dhat
    assert active.sum() > 1e4
    in_contact = np.unique(nodes[active])
    in_contact = in_contact[sc.pinned[in_contact] == 0]
    free = np.flatnonzero(sc.pinned == 0)
    verts = [int(v) for v in np.concatenate([rng.choice(in_contact, 20, replace=False),
                                             rng.choice(free, 4, replace=False)])]
    # oracle rows: elastic + mass, then the contact stencils that touch each vertex
    m = system.make_model(sc)
    ro, go = _oracle_rows(sc, x, verts, mass)
    y = sc.X + sc.h * sc.V0 + sc.h ** 2 * sc.gravity[None, :]
    for v in verts:
        keys = [cand[i] for i in np.flatnonzero(active & np.any(nodes == v, axis=1))]
        if not keys:
            continue
        ps = obal.make_pairset(m, x, keys, {}, sigma)
        _, gc, Hc, nd, _ = contact.contact_terms(x, ps.keys, sc, ps.inA, ps.inAp, ps.mu, ps.s, sigma,
                                                 sc.dhat)
        for k in range(len(ps.keys)):
            a = int(np.flatnonzero(nd[k] == v)[0])
            go[v] = go[v] + gc[k, 3 * a:3 * a + 3]
            for b in range(4):
                u = int(nd[k, b])
                ro[v][u] = ro[v].get(u, np.zeros((3, 3))) + Hc[k, 3 * a:3 * a + 3, 3 * b:3 * b + 3]
    rg = _gpu_rows_with_contact(S, view, verts)
    gg = g.cpu().numpy().reshape(-1, 3)
    for v in verts:
        scale = max(np.abs(B).max() for B in ro[v].values())
        for u, B in ro[v].items():
            if sc.pinned[u]:
                continue
            assert np.abs(rg[v].get(u, np.zeros((3, 3))) - B).max() <= 1e-10 * scale, (v, u)
        for u in rg[v]:                              # no block the oracle does not have
            assert u in ro[v] or np.abs(rg[v][u]).max() <= 1e-10 * scale, (v, u)
        ref = go[v] + mass[v] * (x[v] - y[v]) / sc.h ** 2
        assert np.abs(gg[v] - ref).max() <= 1e-10 * max(np.abs(ref).max(), 1e-30), v
