"""GPU parity: every hot-path call of libbal through the C ABI against the FP64
oracle on the same seeded inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bal as obal  # noqa: E402
from oracle import contact  # noqa: E402
from oracle import system  # noqa: E402
from paper_2407_00046_b300 import bal, scenes  # noqa: E402

from gpu_common import close_cubes, compare_trajectory, gpu_hessian, oracle_state  # noqa: E402

DEV = "cuda"
HESS_TOL = 1e-10      # |H_gpu - H_oracle|_max / |H_oracle|_max
GRAD_TOL = 1e-10


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


@pytest.fixture(scope="module")
def contact_case():
    sc = close_cubes(n=3)
    rng = np.random.default_rng(7)
    x = sc.X + 1e-4 * rng.normal(size=sc.X.shape) * (sc.pinned == 0)[:, None]
    S = bal.Scene(sc, bal.default_params())
    S.step_begin(T(sc.X), T(sc.V0))
    return sc, S, x


def test_sigma0_matches_oracle(contact_case):
    sc, S, _ = contact_case
    m = system.make_model(sc)
    y = system.inertia_target(m, sc.X, sc.V0)
    keys, _ = obal.active_pairs(m, sc.X)
    assert len(keys) > 0
    s0 = obal.initial_sigma(m, sc.X, y, keys)
    al = S.get_al_state()
    assert al["sigma0"] == pytest.approx(s0, rel=1e-10)


@pytest.mark.parametrize("with_ap", [False, True])
def test_assembly_matches_oracle(contact_case, with_ap):
    sc, S, x = contact_case
    sigma = 7.5
    ap = {}
    if with_ap:
        m = system.make_model(sc)
        keys, _ = obal.active_pairs(m, x)
        ap = {k: 0.05 * (i % 5) for i, k in enumerate(keys[::4])}
    S.set_al_state(sigma, sigma, [bal.pair_key(*k) for k in sorted(ap)], [ap[k] for k in sorted(ap)])
    g = torch.empty(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    view = S.assemble_hessian(T(x), g)
    Hg, lam_g, _ = gpu_hessian(S, view)
    m, y, ps = oracle_state(sc, x, sigma, ap)
    # the perturbed lattices put many edge-edge pairs inside the mollified zone
    X4 = x[contact.stencil_nodes(ps.keys, sc)]
    mol = contact.mollifier(X4, contact.ee_eps(ps.keys, sc), derivs=False)
    assert np.sum((mol > 0.0) & (mol < 1.0)) >= 10
    g_or = system.gradient(m, x, y, ps, sigma).ravel()
    H_or, lam_or = system.hessian(m, x, y, ps, sigma, with_lambda=True)
    gerr = np.abs(g.cpu().numpy() - g_or).max() / np.abs(g_or).max()
    herr = np.abs((Hg - H_or).toarray()).max() / np.abs(H_or.toarray()).max()
    lerr = np.abs(lam_g - lam_or).max() / np.abs(lam_or).max()
    assert gerr < GRAD_TOL, gerr
    assert herr < HESS_TOL, herr
    assert lerr < HESS_TOL, lerr
    assert view["nnz_C"] > 0


def test_spmv_matches_oracle(contact_case):
    sc, S, x = contact_case
    S.set_al_state(3.0, 3.0)
    view = S.assemble_hessian(T(x))
    m, y, ps = oracle_state(sc, x, 3.0)
    H_or = system.hessian(m, x, y, ps, 3.0)
    rng = np.random.default_rng(3)
    v = rng.normal(size=3 * sc.n_verts)
    yv = torch.empty_like(T(v))
    S.spmv(T(v), yv)
    ref = H_or @ v
    assert np.abs(yv.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-11
    assert view["nnz_L"] > 0


@pytest.mark.parametrize("tol", [1e-6, 1e-9])
def test_pcg_residual_checked_by_oracle(contact_case, tol):
    sc, S, x = contact_case
    S.set_al_state(3.0, 3.0)
    g = torch.empty(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    S.assemble_hessian(T(x), g)
    m, y, ps = oracle_state(sc, x, 3.0)
    H_or = system.hessian(m, x, y, ps, 3.0)
    b = -g
    sol = torch.zeros_like(b)
    info = S.pcg_solve(b, sol, tol, 5000)
    bn = b.cpu().numpy()
    res = np.linalg.norm(bn - H_or @ sol.cpu().numpy()) / np.linalg.norm(bn)
    assert info["converged"] == 1
    assert res <= 1.05 * tol, (res, info)
    assert abs(info["rel_residual"] - res) <= 1e-3 * res + 1e-15


def test_pcg_edge_cases(contact_case):
    sc, S, x = contact_case
    S.set_al_state(3.0, 3.0)
    S.assemble_hessian(T(x))
    z = torch.zeros(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    sol = torch.zeros_like(z)
    info = S.pcg_solve(z, sol, 1e-8, 100)          # zero right-hand side
    assert info["iters"] == 0 and float(sol.abs().max()) == 0.0
    b = torch.ones_like(z)
    info = S.pcg_solve(b, sol, 1e-8, 0)            # zero iteration cap
    assert info["iters"] == 0


def test_energy_matches_oracle(contact_case):
    sc, S, x = contact_case
    S.set_al_state(4.0, 4.0)
    e = S.energy(T(x))
    m, y, ps = oracle_state(sc, x, 4.0)
    e_or = system.energy(m, x, y, ps, 4.0)
    assert e == pytest.approx(e_or, rel=1e-12)


def test_free_flight_is_exact():
    X, Tt = scenes.lattice_box(3, 3, 3, (0.1, 0.1, 0.1))
    sc = scenes.merge_bodies("free", [dict(X=X, tets=Tt, E=1e5, V0=np.array([0.1, 0.2, -0.3]))])
    S = bal.Scene(sc, bal.default_params(newton_tol=1e-12, pcg_tol=1e-14))
    x, v = T(sc.X), T(sc.V0)
    S.step_begin(x, v)
    y = torch.empty_like(x)
    S.get_y(y)
    info = S.time_step(x, v)
    assert info["converged"] == 1
    assert float((x - y).abs().max()) < 1e-13


def test_time_step_trajectory_small():
    sc = close_cubes(n=2, gap=5e-4)
    S = bal.Scene(sc, bal.default_params(newton_tol=1e-8, pcg_tol=1e-12, pcg_max_iter=20000))
    m = system.make_model(sc)
    assert compare_trajectory(S, m, sc, 3, obal.Params(newton_tol=1e-8), T) >= 1


def test_newton_step_counts_match_oracle():
    sc = close_cubes(n=2, gap=3e-4)
    S = bal.Scene(sc, bal.default_params(newton_tol=1e-8, pcg_tol=1e-12))
    x, v = T(sc.X), T(sc.V0)
    S.step_begin(x, v)
    info = S.newton_step(x)
    m = system.make_model(sc)
    keys, _ = obal.active_pairs(m, sc.X)
    assert info["n_active"] == len(keys) and info["n_active"] > 0
    assert info["alpha"] > 0


@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_mixed_precision_pcg_refines_to_fp64_residual(contact_case, tol):
    # FP32 SpMV / preconditioner inside, FP64 residual outside (iterative refinement)
    sc, S, x = contact_case
    S.set_al_state(3.0, 3.0)
    g = torch.empty(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    S.assemble_hessian(T(x), g)
    m, y, ps = oracle_state(sc, x, 3.0)
    H_or = system.hessian(m, x, y, ps, 3.0)
    S.set_params(precision=bal.PREC_MIXED, mixed_inner_tol=1e-4, mixed_max_refine=30)
    try:
        b = -g
        sol = torch.zeros_like(b)
        info = S.pcg_solve(b, sol, tol, 20000)
    finally:
        S.set_params(precision=bal.PREC_FP64)
    bn = b.cpu().numpy()
    res = np.linalg.norm(bn - H_or @ sol.cpu().numpy()) / np.linalg.norm(bn)
    assert info["converged"] == 1 and info["refine_passes"] >= 1
    assert res <= 1.05 * tol, (res, info)


def test_mixed_precision_trajectory_matches_oracle():
    sc = close_cubes(n=2, gap=5e-4)
    S = bal.Scene(sc, bal.default_params(newton_tol=1e-8, pcg_tol=1e-12, pcg_max_iter=20000,
                                         precision=bal.PREC_MIXED, mixed_inner_tol=1e-4,
                                         mixed_max_refine=40))
    m = system.make_model(sc)
    compare_trajectory(S, m, sc, 2, obal.Params(newton_tol=1e-8), T)


def test_warm_start_solves_the_grouped_system(contact_case):
    # warm start alone (global PCG given no iterations): the subdomain solve on
    # H_dom (blocks coupling different floor(log10 e_j) groups removed)
    import scipy.sparse.linalg as spla
    sc, S, x = contact_case
    S.set_al_state(3.0, 3.0)
    g = torch.empty(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    S.assemble_hessian(T(x), g)
    m, y, ps = oracle_state(sc, x, 3.0)
    H_or, lam = system.hessian(m, x, y, ps, 3.0, with_lambda=True)
    e, grp = system.groups_from_lambda(lam)
    frac = np.abs(np.log10(e) - np.round(np.log10(e)))
    assert frac.min() > 1e-9          # no node sits on a group boundary
    Hd = system.masked_hessian(H_or, grp)
    b = -g
    S.set_params(precond=bal.PRECOND_BJ_WARMSTART, warm_tol=1e-13, warm_max_iter=5000)
    try:
        sol = torch.zeros_like(b)
        info = S.pcg_solve(b, sol, 1e-8, 0)
        ref = spla.spsolve(Hd.tocsc(), b.cpu().numpy())
        assert info["n_groups"] == len(np.unique(grp))
        err = np.abs(sol.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err < 1e-9, err
        # full solve: warm start then global PCG to tolerance
        S.set_params(warm_tol=1e-2, warm_max_iter=50)
        sol.zero_()
        info = S.pcg_solve(b, sol, 1e-9, 5000)
        bn = b.cpu().numpy()
        res = np.linalg.norm(bn - H_or @ sol.cpu().numpy()) / np.linalg.norm(bn)
        assert info["converged"] == 1 and info["warm_iters"] > 0
        # the global PCG tolerance is relative to its own r_0 (after the warm start)
        r0_over_b = info["rel_residual"] / info["rel_residual_r0"]
        assert res <= 1.05e-9 * max(1.0, r0_over_b), (res, info)
    finally:
        S.set_params(precond=bal.PRECOND_BJ)


def _fine_on_coarse():
    """A 6^3-cell cube (small vertex ids) resting 0.4 mm above the top face of a
    single-cell box (large vertex ids): every point of the fine bottom face
    is in contact with one of two big triangles, so the rows of the box's
    top vertices collect many emitted blocks (more than 32) with long runs of
    the same column."""
    from paper_2407_00046_b300.scenes import lattice_box, merge_bodies
    Xf, Tf = lattice_box(6, 6, 6, (0.03, 0.03, 0.03))
    Xc, Tc = lattice_box(1, 1, 1, (0.06, 0.02, 0.06))
    Xf = Xf + np.array([0.012, 0.0204, 0.012])
    rng = np.random.default_rng(4)
    Xf = Xf + 2e-5 * rng.normal(size=Xf.shape)
    return merge_bodies("fine_on_coarse", [dict(X=Xf, tets=Tf, E=1e5),
                                           dict(X=Xc, tets=Tc, E=1e6,
                                                pinned=Xc[:, 1] <= 1e-12)])


def test_contact_merge_with_long_rows_matches_oracle():
    sc = _fine_on_coarse()
    m = system.make_model(sc)
    keys, d = obal.active_pairs(m, sc.X)
    assert len(keys) > 40 and d.min() > 0
    S = bal.Scene(sc, bal.default_params())
    S.step_begin(T(sc.X), T(sc.V0))
    sigma = 2.0
    S.set_al_state(sigma, sigma)
    g = torch.empty(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    view = S.assemble_hessian(T(sc.X), g)
    Hg, _, parts = gpu_hessian(S, view)
    # rows of the coarse box with more than 32 contact records (6 emitted per pair)
    nodes = contact.stencil_nodes(keys, sc)
    emitted = {}
    for st in nodes:
        for a in range(4):
            for b in range(a):
                r, c = max(st[a], st[b]), min(st[a], st[b])
                if r != c and not (sc.pinned[r] or sc.pinned[c]):
                    emitted[r] = emitted.get(r, 0) + 1
    assert max(emitted.values()) > 64
    # C sorted by (row, col) without duplicates
    rc = parts["Cr"].astype(np.int64) * sc.n_verts + parts["Cc"]
    assert np.all(np.diff(rc) > 0) and np.all(parts["Cr"] > parts["Cc"])
    y = system.inertia_target(m, sc.X, sc.V0)
    ps = obal.make_pairset(m, sc.X, keys, {}, sigma)
    H_or = system.hessian(m, sc.X, y, ps, sigma)
    herr = np.abs((Hg - H_or).toarray()).max() / np.abs(H_or.toarray()).max()
    assert herr < HESS_TOL, herr
    # bit-reproducible merge: a second assembly gives identical blocks
    view2 = S.assemble_hessian(T(sc.X), g)
    _, _, parts2 = gpu_hessian(S, view2)
    assert np.array_equal(parts["Cv"], parts2["Cv"]) and np.array_equal(parts["Cr"], parts2["Cr"])
