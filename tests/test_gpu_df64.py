"""GPU parity of the double-float PCG (BAL_PREC_DF64) through the C ABI: the
first CG iterates against a textbook block-Jacobi CG on the oracle's Hessian
(so the gather SpMV, static blocks both ways and contact blocks both ways, is
checked element by element), the FP64 residual of full solves, determinism, the
FP64 fallback for entries beyond the FP32 range, and a trajectory."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bal as obal  # noqa: E402
from oracle import system  # noqa: E402
from paper_2407_00046_b300 import bal, scenes  # noqa: E402

from gpu_common import close_cubes, compare_trajectory, oracle_state  # noqa: E402

DEV = "cuda"


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


@pytest.fixture(scope="module")
def multi_tile_case():
    # 686 vertices: 22 slices of 32 rows, the last one ragged; contact blocks present
    sc = close_cubes(n=6)
    rng = np.random.default_rng(11)
    x = sc.X + 1e-4 * rng.normal(size=sc.X.shape) * (sc.pinned == 0)[:, None]
    S = bal.Scene(sc, bal.default_params())
    S.step_begin(T(sc.X), T(sc.V0))
    S.set_al_state(3.0, 3.0)
    g = torch.empty(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    view = S.assemble_hessian(T(x), g)
    assert view["nnz_C"] > 0 and sc.n_verts % 32 != 0 and sc.n_verts > 512
    m, y, ps = oracle_state(sc, x, 3.0)
    H = system.hessian(m, x, y, ps, 3.0).tocsr()
    return sc, S, x, -g, H, m, y


def _permuted(sc, seed):
    """The same scene with its vertex ids shuffled (no lattice ordering left)."""
    import copy
    rng = np.random.default_rng(seed)
    perm = rng.permutation(sc.n_verts)           # new id of old vertex v is perm[v]
    inv = np.argsort(perm)
    out = copy.deepcopy(sc)
    for name in ("X", "V0", "pinned", "body"):
        setattr(out, name, getattr(sc, name)[inv])
    out.tets = perm[sc.tets].astype(np.int32)
    out.tris = perm[sc.tris].astype(np.int32)
    out.edges = np.sort(perm[sc.edges], axis=1).astype(np.int32)
    out.surf_verts = np.sort(perm[sc.surf_verts]).astype(np.int32)
    return out


def test_df64_iterates_on_shuffled_vertex_order():
    sc = _permuted(close_cubes(n=6), 5)
    rng = np.random.default_rng(12)
    x = sc.X + 1e-4 * rng.normal(size=sc.X.shape) * (sc.pinned == 0)[:, None]
    S = bal.Scene(sc, bal.default_params(precision=bal.PREC_DF64, pcg_stall_window=0))
    S.step_begin(T(sc.X), T(sc.V0))
    S.set_al_state(3.0, 3.0)
    g = torch.empty(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    view = S.assemble_hessian(T(x), g)
    assert view["nnz_C"] > 0
    m, y, ps = oracle_state(sc, x, 3.0)
    H = system.hessian(m, x, y, ps, 3.0).tocsr()
    ref = _block_jacobi_cg(H, -g.cpu().numpy(), 3)
    sol = torch.zeros_like(g)
    info = S.pcg_solve(-g, sol, 1e-30, 3)
    assert info["iters"] == 3
    assert np.abs(sol.cpu().numpy() - ref).max() <= 1e-11 * np.abs(ref).max()


def _block_jacobi_cg(H, b, iters):
    """Textbook PCG (x0 = 0) with the inverse 3x3 diagonal blocks of H."""
    n = b.size // 3
    Hd = H.toarray() if n <= 2000 else None
    Dinv = np.stack([np.linalg.inv(Hd[3 * i:3 * i + 3, 3 * i:3 * i + 3]) for i in range(n)])
    prec = lambda r: np.einsum("nij,nj->ni", Dinv, r.reshape(n, 3)).ravel()  # noqa: E731
    x = np.zeros_like(b)
    r = b.copy()
    z = prec(r)
    p = z.copy()
    rz = r @ z
    for _ in range(iters):
        q = H @ p
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        z = prec(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x


def _diag_block_inverses(H, n):
    C = H.tocoo()
    keep = (C.row // 3) == (C.col // 3)
    B = np.zeros((n, 3, 3))
    np.add.at(B, (C.row[keep] // 3, C.row[keep] % 3, C.col[keep] % 3), C.data[keep])
    return np.linalg.inv(B)


def test_df64_iterates_across_sorting_windows():
    """5,488 vertices: two windows of the slot sort (4,096 + a ragged 1,392)
    and a ragged last slice; three df64 PCG iterates against textbook
    block-Jacobi CG on the oracle's Hessian."""
    sc = scenes.cube_stack(n_cubes=2, n=13)
    assert sc.n_verts > 4096 and sc.n_verts % 4096 != 0 and sc.n_verts % 32 != 0
    rng = np.random.default_rng(14)
    x = sc.X + 2e-4 * rng.normal(size=sc.X.shape) * (sc.pinned == 0)[:, None]
    S = bal.Scene(sc, bal.default_params(precision=bal.PREC_DF64, pcg_stall_window=0))
    S.step_begin(T(sc.X), T(sc.V0))
    S.set_al_state(3.0, 3.0)
    g = torch.empty(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    S.assemble_hessian(T(x), g)
    m, y, ps = oracle_state(sc, x, 3.0)
    H = system.hessian(m, x, y, ps, 3.0).tocsr()
    n = sc.n_verts
    Dinv = _diag_block_inverses(H, n)
    prec = lambda r: np.einsum("nij,nj->ni", Dinv, r.reshape(n, 3)).ravel()  # noqa: E731
    b = -g.cpu().numpy()
    xr, r = np.zeros_like(b), b.copy()
    z = prec(r)
    p, rz = z.copy(), r @ z
    for _ in range(3):
        q = H @ p
        a = rz / (p @ q)
        xr += a * p
        r -= a * q
        z = prec(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    sol = torch.zeros_like(g)
    info = S.pcg_solve(-g, sol, 1e-30, 3)
    assert info["iters"] == 3 and info["precision_used"] == bal.PREC_DF64
    assert np.abs(sol.cpu().numpy() - xr).max() <= 1e-11 * np.abs(xr).max()


@pytest.mark.parametrize("iters", [1, 2, 5])
def test_df64_iterates_match_textbook_cg_on_oracle_hessian(multi_tile_case, iters):
    sc, S, x, b, H, m, y = multi_tile_case
    ref = _block_jacobi_cg(H, b.cpu().numpy(), iters)
    # without contact blocks the iterate moves by far more than the tolerance
    H_nc = system.hessian(m, x, y, obal.make_pairset(m, x, [], {}, 3.0), 3.0).tocsr()
    ref_nc = _block_jacobi_cg(H_nc, b.cpu().numpy(), iters)
    scale = np.abs(ref).max()
    assert np.abs(ref - ref_nc).max() > 1e-6 * scale
    S.set_params(precision=bal.PREC_DF64, pcg_stall_window=0)
    try:
        sol = torch.zeros_like(b)
        info = S.pcg_solve(b, sol, 1e-30, iters)
    finally:
        S.set_params(precision=bal.PREC_FP64, pcg_stall_window=100)
    assert info["iters"] == iters and info["precision_used"] == bal.PREC_DF64
    err = np.abs(sol.cpu().numpy() - ref).max() / scale
    assert err < 1e-11, err


@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_df64_pcg_reaches_fp64_residual(multi_tile_case, tol):
    sc, S, x, b, H, m, y = multi_tile_case
    S.set_params(precision=bal.PREC_DF64)
    try:
        sol = torch.zeros_like(b)
        info = S.pcg_solve(b, sol, tol, 20000)
    finally:
        S.set_params(precision=bal.PREC_FP64)
    bn = b.cpu().numpy()
    res = np.linalg.norm(bn - H @ sol.cpu().numpy()) / np.linalg.norm(bn)
    assert info["converged"] == 1 and info["precision_used"] == bal.PREC_DF64
    assert res <= 1.05 * tol, (res, info)
    assert abs(info["rel_residual"] - res) <= 1e-3 * res + 1e-15
    # same iteration count as the FP64 solver up to rounding-driven drift
    sol64 = torch.zeros_like(b)
    info64 = S.pcg_solve(b, sol64, tol, 20000)
    assert abs(info["iters"] - info64["iters"]) <= max(3, 0.05 * info64["iters"]), (info, info64)


def test_df64_pcg_is_deterministic(multi_tile_case):
    sc, S, x, b, H, m, y = multi_tile_case
    S.set_params(precision=bal.PREC_DF64)
    try:
        outs = []
        for _ in range(2):
            sol = torch.zeros_like(b)
            S.pcg_solve(b, sol, 1e-8, 5000)
            outs.append(sol.clone())
    finally:
        S.set_params(precision=bal.PREC_FP64)
    assert torch.equal(outs[0], outs[1])


def test_df64_edge_cases(multi_tile_case):
    sc, S, x, b, H, m, y = multi_tile_case
    S.set_params(precision=bal.PREC_DF64)
    try:
        z = torch.zeros_like(b)
        sol = torch.zeros_like(b)
        info = S.pcg_solve(z, sol, 1e-8, 100)       # zero right-hand side
        assert info["iters"] == 0 and float(sol.abs().max()) == 0.0
        info = S.pcg_solve(b, sol, 1e-8, 0)         # zero iteration cap
        assert info["iters"] == 0 and float(sol.abs().max()) == 0.0
        # non-zero start: the tolerance is relative to the residual at x0
        x0 = torch.zeros_like(b)
        S.set_params(precision=bal.PREC_FP64)
        S.pcg_solve(b, x0, 1e-3, 20000)
        S.set_params(precision=bal.PREC_DF64)
        r0 = np.linalg.norm(b.cpu().numpy() - H @ x0.cpu().numpy())
        info = S.pcg_solve(b, x0, 1e-6, 20000)
        res = np.linalg.norm(b.cpu().numpy() - H @ x0.cpu().numpy())
        assert info["converged"] == 1 and res <= 1.05e-6 * r0
    finally:
        S.set_params(precision=bal.PREC_FP64)


def test_df64_falls_back_to_fp64_beyond_fp32_range():
    X, Tt = scenes.lattice_box(2, 2, 2, (0.01, 0.01, 0.01))
    sc = scenes.merge_bodies("stiff", [dict(X=X, tets=Tt, E=1e44, V0=np.zeros(3))])
    S = bal.Scene(sc, bal.default_params(precision=bal.PREC_DF64))
    rng = np.random.default_rng(2)
    x = sc.X + 1e-4 * rng.normal(size=sc.X.shape)
    S.step_begin(T(sc.X), T(sc.V0))
    g = torch.empty(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    S.assemble_hessian(T(x), g)
    sol = torch.zeros_like(g)
    info = S.pcg_solve(-g, sol, 1e-8, 5000)
    assert info["precision_used"] == bal.PREC_FP64 and info["converged"] == 1


def test_df64_trajectory_matches_oracle():
    sc = close_cubes(n=2, gap=5e-4)
    S = bal.Scene(sc, bal.default_params(newton_tol=1e-8, pcg_tol=1e-12, pcg_max_iter=20000,
                                         precision=bal.PREC_DF64))
    m = system.make_model(sc)
    compare_trajectory(S, m, sc, 2, obal.Params(newton_tol=1e-8), T)


def _textbook_iterates(H, b, n, iters):
    Dinv = _diag_block_inverses(H, n)
    prec = lambda r: np.einsum("nij,nj->ni", Dinv, r.reshape(n, 3)).ravel()  # noqa: E731
    xr, r = np.zeros_like(b), b.copy()
    z = prec(r)
    p, rz = z.copy(), r @ z
    for _ in range(iters):
        q = H @ p
        a = rz / (p @ q)
        xr += a * p
        r -= a * q
        z = prec(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return xr


@pytest.mark.parametrize("case,window", [("stack", 32), ("stack", 512), ("stack", 1024),
                                         ("shuffled", 64), ("shuffled", 4096), ("contact", 256)])
def test_df64_windowed_spmv_iterates(case, window):
    """The windowed SpMV layout (one CTA per window of rows, in-window transposes
    summed in shared memory, the rest through the column-side list): three
    iterates against textbook block-Jacobi CG on the oracle's Hessian, with
    several windows and a ragged last one (5,488-vertex two-cube stack), a
    shuffled vertex order (most transposes cross windows), and contact blocks.
    The shared sums are FP64 in arrival order, so the bar is the df64 one."""
    if case == "stack":
        sc = scenes.cube_stack(n_cubes=2, n=13)
        sigma, noise = 3.0, 2e-4
    elif case == "shuffled":
        sc, sigma, noise = _permuted(close_cubes(n=6), 7), 3.0, 1e-4
    else:
        sc, sigma, noise = close_cubes(n=6), 3.0, 1e-4
    rng = np.random.default_rng(15)
    x = sc.X + noise * rng.normal(size=sc.X.shape) * (sc.pinned == 0)[:, None]
    S = bal.Scene(sc, bal.default_params(precision=bal.PREC_DF64, pcg_stall_window=0, spmv_window=window))
    S.step_begin(T(sc.X), T(sc.V0))
    S.set_al_state(sigma, sigma)
    g = torch.empty(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    view = S.assemble_hessian(T(x), g)
    if case == "contact":
        assert view["nnz_C"] > 0
    m, y, ps = oracle_state(sc, x, sigma)
    H = system.hessian(m, x, y, ps, sigma).tocsr()
    ref = _textbook_iterates(H, -g.cpu().numpy(), sc.n_verts, 3)
    sol = torch.zeros_like(g)
    info = S.pcg_solve(-g, sol, 1e-30, 3)
    assert info["iters"] == 3 and info["precision_used"] == bal.PREC_DF64
    assert np.abs(sol.cpu().numpy() - ref).max() <= 1e-11 * np.abs(ref).max()
    # a full solve reaches the FP64 residual
    sol.zero_()
    S.set_params(pcg_stall_window=1000)
    info = S.pcg_solve(-g, sol, 1e-8, 20000)
    bn = -g.cpu().numpy()
    res = np.linalg.norm(bn - H @ sol.cpu().numpy()) / np.linalg.norm(bn)
    assert info["converged"] == 1 and res <= 1.05e-8, (res, info)


@pytest.mark.parametrize("precision", [bal.PREC_DF64, bal.PREC_FP64])
def test_stagnation_window_obeys_the_forcing_bound(multi_tile_case, precision):
    """With a one-iteration stagnation window a solve stops at the first
    iteration that does not improve sqrt(r^T z); with the forcing bound
    eta = 0.5 it may stop that way only once ||r|| <= 0.5 ||r_0||."""
    sc, S, x, b, H, m, y = multi_tile_case
    bn = b.cpu().numpy()
    out = {}
    try:
        for eta in (0.0, 0.5):
            S.set_params(precision=precision, pcg_stall_window=1, pcg_stall_forcing=eta)
            sol = torch.zeros_like(b)
            info = S.pcg_solve(b, sol, 1e-12, 5000)
            res = np.linalg.norm(bn - H @ sol.cpu().numpy()) / np.linalg.norm(bn)
            out[eta] = (info, res)
    finally:
        S.set_params(precision=bal.PREC_FP64, pcg_stall_window=100, pcg_stall_forcing=0.0)
    info, res = out[0.5]
    assert info["converged"] == 1 or info["iters"] == 5000 or res <= 0.5 * 1.001, (info, res)
    assert out[0.5][0]["iters"] >= out[0.0][0]["iters"]
