"""The first Newton direction of the 1,053,696-tet stack of 64 cubes (4 x 4
columns of 4, n = 14, E log-uniform in [1e5, 1e9] per cube), GPU against the
oracle's exact sparse LU solve of its own assembled system (Sec. 3.1 step
objective at x = x_t, no contact yet; Sec. 4.2.2 projected Hessian; the PCG of
Sec. 4.2 with block-Jacobi).

What is checked, per solver form:
- the GPU direction p solves the ORACLE's system H p = b (its Hessian and its
  b = -grad L, both assembled in FP64 on the CPU) to the PCG tolerance:
  ||b - H p|| <= c * tol * ||b||. This covers the GPU's gradient, Hessian
  assembly and solve at once.
- the direction error that follows: every eigenvalue of the pinned-eliminated
  H is at least lambda_lb = min over free vertices of m_v / h^2 (the elastic
  part is PSD after projection, pinned rows carry m_v / h^2), so
  ||p - p*||_2 <= ||b - H p||_2 / lambda_lb for the exact solution p*. With
  the LU solution's own residual r_LU,
  ||p - p_LU||_2 <= (||b - H p|| + ||r_LU||) / lambda_lb; this bounds the
  largest per-vertex difference too.

The FP32 + FP64-refinement form (FP32 operator in difference form) is held to
the same bound when it reports convergence; otherwise (kappa of the 1e9 cubes
against the FP32 epsilon) it must at least return a direction whose residual
is no larger than ||b|| (a refinement pass that raises the FP64 residual is
rolled back)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bal as obal  # noqa: E402
from oracle import system  # noqa: E402
from paper_2407_00046_b300 import bal, scenes  # noqa: E402

TOL = 1e-6
# Block-Jacobi leaves the rigid modes of the free 1e9 Pa cubes at eigenvalues
# (m_v / h^2) / K_diag ~ 4e-8 of D^-1 H, so kappa ~ 5e7 and CG needs on the
# order of sqrt(kappa) ln(2 / tol) ~ 1e5 iterations; the mixed form restarts
# CG on every refinement pass, and rounding the FP32 vectors still perturbs
# the cubes' rotation modes by O(kappa eps_32), so its cap only bounds the
# test's time.
MAX_ITER = {"fp64": 200000, "df64": 200000, "mixed": 100000}


@pytest.fixture(scope="module")
def oracle_system():
    sc = scenes.cube_columns()
    t0 = time.perf_counter()
    model = system.make_model(sc)
    y = system.inertia_target(model, sc.X, sc.V0)
    ps = system.empty_pairs()
    e = system.gradient(model, sc.X, y, ps, 0.0).ravel()
    H = system.hessian(model, sc.X, y, ps, 0.0)
    t1 = time.perf_counter()
    p_lu = obal.solve(H, -e)
    t2 = time.perf_counter()
    r_lu = float(np.linalg.norm(-e - H @ p_lu))
    lam_lb = float((model.mass[model.free] / model.h ** 2).min())
    print(f"\n[oracle] assembly {t1 - t0:.1f} s, SuperLU {t2 - t1:.1f} s, "
          f"|r_LU|/|b| {r_lu / np.linalg.norm(e):.2e}, lambda_lb {lam_lb:.4g}")
    return sc, e, H, p_lu, r_lu, lam_lb


@pytest.fixture(scope="module")
def gpu_scene(oracle_system):
    sc = oracle_system[0]
    S = bal.Scene(sc, bal.default_params(pcg_stall_window=20000, pcg_max_iter=MAX_ITER["fp64"]),
                  pair_capacity=1 << 22)
    x0 = torch.tensor(sc.X, dtype=torch.float64, device="cuda").contiguous()
    v0 = torch.tensor(sc.V0, dtype=torch.float64, device="cuda").contiguous()
    S.step_begin(x0, v0)
    g = torch.empty_like(x0)
    view = S.assemble_hessian(x0, g)
    assert view["nnz_C"] == 0
    return S, g.view(-1)


@pytest.mark.parametrize("form", ["fp64", "df64", "mixed"])
def test_first_newton_direction_matches_superlu(oracle_system, gpu_scene, form):
    sc, e, H, p_lu, r_lu, lam_lb = oracle_system
    S, g = gpu_scene
    prec = {"fp64": bal.PREC_FP64, "df64": bal.PREC_DF64, "mixed": bal.PREC_MIXED}[form]
    S.set_params(precision=prec, pcg_stall_window=20000, pcg_max_iter=MAX_ITER[form], mixed_inner_max=3000,
                 mixed_max_refine=60, mixed_inner_tol=1e-2)
    sol = torch.zeros_like(g)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = S.pcg_solve(-g, sol, TOL, MAX_ITER[form])
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    p = sol.cpu().numpy()
    assert np.isfinite(p).all()
    b = -e
    bn = float(np.linalg.norm(b))
    r = float(np.linalg.norm(b - H @ p))
    diff = p - p_lu
    dv = float(np.linalg.norm(diff.reshape(-1, 3), axis=1).max())
    print(f"\n[{form}] iters {info['iters']} passes {info['refine_passes']} converged "
          f"{info['converged']} {sec:.2f} s; true rel residual {r / bn:.3e}; "
          f"|p - p_LU|_2 {np.linalg.norm(diff):.3e} (bound {(r + r_lu) / lam_lb:.3e}); "
          f"max per-vertex {dv:.3e} m of max |p_v| {np.abs(p_lu).max():.3e} m")
    if form != "mixed" or info["converged"]:
        assert info["converged"] == 1
        # the FP64 recursion's residual drifts from the true one by a few
        # tolerances at this conditioning; the df64 form restarts on the true one
        c = 1.01 if form == "df64" else 4.0
        assert r <= c * TOL * bn, (r / bn, c * TOL)
        bound = (c * TOL * bn + r_lu) / lam_lb
        assert np.linalg.norm(diff) <= bound
        assert dv <= bound
    else:
        assert r <= bn * (1 + 1e-12)
