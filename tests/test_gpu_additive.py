"""GPU parity of the two-level additive preconditioner (App. A, the paper's
comparison): the first PCG iterates against a textbook PCG on the oracle's
Hessian with M^{-1} = D^{-1} + sum_g B_g^T H_gg^{-1} B_g (groups of 9
consecutive vertices, the last one ragged), and a solve to tolerance."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import system  # noqa: E402
from paper_2407_00046_b300 import bal  # noqa: E402

from gpu_common import close_cubes, oracle_state  # noqa: E402

DEV = "cuda"
GROUP = 9


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


@pytest.fixture(scope="module")
def case():
    sc = close_cubes(n=6)                        # 686 vertices: 76 full groups and one of 2
    rng = np.random.default_rng(13)
    x = sc.X + 1e-4 * rng.normal(size=sc.X.shape) * (sc.pinned == 0)[:, None]
    S = bal.Scene(sc, bal.default_params(precond=bal.PRECOND_ADDITIVE, pcg_stall_window=0))
    S.step_begin(T(sc.X), T(sc.V0))
    S.set_al_state(3.0, 3.0)
    g = torch.empty(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    view = S.assemble_hessian(T(x), g)
    assert view["nnz_C"] > 0 and sc.n_verts % GROUP != 0
    m, y, ps = oracle_state(sc, x, 3.0)
    H = system.hessian(m, x, y, ps, 3.0).toarray()
    return sc, S, -g, H


def _additive_inverse(H):
    n = H.shape[0] // 3
    Minv = np.zeros_like(H)
    for i in range(n):
        s = slice(3 * i, 3 * i + 3)
        Minv[s, s] += np.linalg.inv(H[s, s])
    for g0 in range(0, n, GROUP):
        s = slice(3 * g0, 3 * min(g0 + GROUP, n))
        Minv[s, s] += np.linalg.inv(H[s, s])
    return Minv


def _pcg(H, Minv, b, iters):
    x = np.zeros_like(b)
    r = b.copy()
    z = Minv @ r
    p = z.copy()
    rz = r @ z
    for _ in range(iters):
        q = H @ p
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        z = Minv @ r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x


@pytest.mark.parametrize("iters", [1, 3, 8])
def test_additive_iterates_match_textbook_pcg(case, iters):
    sc, S, b, H = case
    Minv = _additive_inverse(H)
    ref = _pcg(H, Minv, b.cpu().numpy(), iters)
    sol = torch.zeros_like(b)
    info = S.pcg_solve(b, sol, 1e-30, iters)
    assert info["iters"] == iters and info["precision_used"] == bal.PREC_FP64
    err = np.abs(sol.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 1e-10, err


def test_additive_solve_reaches_tolerance(case):
    sc, S, b, H = case
    sol = torch.zeros_like(b)
    info = S.pcg_solve(b, sol, 1e-9, 20000)
    bn = b.cpu().numpy()
    res = np.linalg.norm(bn - H @ sol.cpu().numpy()) / np.linalg.norm(bn)
    assert info["converged"] == 1 and res <= 1.05e-9, (res, info)
