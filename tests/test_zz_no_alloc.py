"""The allocation-free PCG entry point (bal_pcg_solve_noalloc), for callers
that cannot allocate GPU memory while they run, gives the same solution as the
regular bal_pcg_solve on the same assembled Hessian, on two calls in a row
(its fixed scratch array keeps the previous call's contents, which must not
leak into the next). Collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2407_00046_b300 import bal  # noqa: E402

from gpu_common import close_cubes  # noqa: E402

TOL = 1e-10


def _assembled():
    sc = close_cubes(n=3)
    rng = np.random.default_rng(11)
    x = sc.X + 1e-4 * rng.normal(size=sc.X.shape) * (sc.pinned == 0)[:, None]
    S = bal.Scene(sc, bal.default_params())
    dev = torch.device("cuda")
    S.step_begin(torch.tensor(sc.X, dtype=torch.float64, device=dev),
                 torch.tensor(sc.V0, dtype=torch.float64, device=dev))
    S.set_al_state(5.0, 5.0)
    view = S.assemble_hessian(torch.tensor(x, dtype=torch.float64, device=dev))
    h = S.copy_hessian(view)
    rp, col = S.static_pattern()
    rows_L = np.repeat(np.arange(S.nv), np.diff(rp)).astype(np.int32)
    rows = torch.cat([torch.tensor(rows_L, device=dev), h["C_row"]]).contiguous()
    cols = torch.cat([torch.tensor(col, device=dev), h["C_col"]]).contiguous()
    vals = torch.cat([h["L"], h["C_val"]]).contiguous()
    return S, h["D"].contiguous(), rows, cols, vals


def test_noalloc_matches_regular_solve_twice():
    S, D, rows, cols, vals = _assembled()
    n = 3 * S.nv
    gen = torch.Generator(device="cuda").manual_seed(5)
    for call in range(2):
        b = torch.randn(n, dtype=torch.float64, device="cuda", generator=gen)
        ref = torch.zeros_like(b)
        info_ref = S.pcg_solve(b, ref, TOL, 20000)
        sol = torch.zeros_like(b)
        info = bal.pcg_solve_noalloc(D, rows, cols, vals, b, sol, TOL, 20000)
        assert info["converged"] == 1 and info_ref["converged"] == 1, (call, info, info_ref)
        assert info["rel_residual"] <= 1.05 * TOL
        rel = float((sol - ref).norm() / ref.norm())
        assert rel < 1e-6, (call, rel)
        # residual of the no-alloc solution measured with the regular SpMV
        hx = torch.empty_like(b)
        S.spmv(sol, hx)
        assert float((b - hx).norm() / b.norm()) <= 1.05 * TOL


def test_noalloc_rejects_sizes_beyond_its_limit():
    n = bal.NOALLOC_MAX_VERTS + 1
    D = torch.zeros(9 * n, dtype=torch.float64, device="cuda")
    v = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    with pytest.raises(bal.BalError, match="BAL_NOALLOC_MAX_VERTS"):
        bal.pcg_solve_noalloc(D, e, e, torch.zeros(0, dtype=torch.float64, device="cuda"), v, v,
                              1e-8, 10)


def test_noalloc_warm_start_cap_empty_lower_part_and_singular_block():
    """A nonzero initial guess and an iteration cap give the regular solve's
    iterate; a matrix without lower blocks solves block by block; a singular
    diagonal block is reported as BAL_ERR_NAN."""
    S, D, rows, cols, vals = _assembled()
    n = 3 * S.nv
    gen = torch.Generator(device="cuda").manual_seed(9)
    b = torch.randn(n, dtype=torch.float64, device="cuda", generator=gen)
    x0 = 1e-3 * torch.randn(n, dtype=torch.float64, device="cuda", generator=gen)
    # warm start to convergence
    ref, sol = x0.clone(), x0.clone()
    info_ref = S.pcg_solve(b, ref, TOL, 20000)
    info = bal.pcg_solve_noalloc(D, rows, cols, vals, b, sol, TOL, 20000)
    assert info["converged"] == 1 and info_ref["converged"] == 1
    assert float((sol - ref).norm() / ref.norm()) < 1e-6
    # iteration cap: the same count and nearly the same iterate (atomic sums differ in rounding)
    ref, sol = x0.clone(), x0.clone()
    info_ref = S.pcg_solve(b, ref, 1e-14, 7)
    info = bal.pcg_solve_noalloc(D, rows, cols, vals, b, sol, 1e-14, 7)
    assert info["iters"] == info_ref["iters"] == 7 and info["converged"] == 0
    assert float((sol - ref).norm() / ref.norm()) < 1e-9
    # no lower blocks: H = D, one PCG iteration solves each 3x3 system
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    ev = torch.zeros(0, dtype=torch.float64, device="cuda")
    sol = torch.zeros_like(b)
    info = bal.pcg_solve_noalloc(D, e, e, ev, b, sol, 1e-12, 10)
    assert info["converged"] == 1 and info["iters"] <= 1
    Db = D.view(-1, 3, 3)
    res = b.view(-1, 3) - torch.einsum("nij,nj->ni", Db, sol.view(-1, 3))
    assert float(res.norm() / b.norm()) <= 1e-12
    # a singular diagonal block: D^-1 is not finite
    Ds = D.clone()
    Ds[:9] = 0.0
    with pytest.raises(bal.BalError, match="NAN"):
        bal.pcg_solve_noalloc(Ds, e, e, ev, b, torch.zeros_like(b), 1e-12, 10)
