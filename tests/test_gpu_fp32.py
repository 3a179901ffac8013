"""GPU parity of the single-precision path (BAL_PREC_FP32): element stencil
eigensystems in FP32, FP32 PCG with FP64 refinement, FP64 gradient, contact
and energies.

Tolerances. The FP32 element Hessian goes through ~10^3 FP32 operations per
block (SVD by Jacobi, the 3x3 scaling eigenproblem, 9 rank-one updates) with
unit roundoff u = 6e-8; a bound of 5e-5 of the largest entry leaves a margin
of ~10 over u times that operation count's square root times the element
condition. The gradient is FP64 (1e-10, as the FP64 path). The time step's
end state is decided by the FP64 gradient's convergence test, so it carries
the FP64 path's 1e-8 m."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bal as obal  # noqa: E402
from oracle import system  # noqa: E402
from paper_2407_00046_b300 import bal  # noqa: E402

from gpu_common import close_cubes, compare_trajectory, gpu_hessian, oracle_state  # noqa: E402

DEV = "cuda"
HESS_TOL_F32 = 5e-5


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


@pytest.mark.parametrize("amp", [1e-4, 3e-3])
def test_fp32_element_hessian_within_fp32_tolerance(amp):
    sc = close_cubes(n=3)
    rng = np.random.default_rng(17)
    x = sc.X + amp * rng.normal(size=sc.X.shape) * (sc.pinned == 0)[:, None]
    S = bal.Scene(sc, bal.default_params(precision=bal.PREC_FP32))
    S.step_begin(T(sc.X), T(sc.V0))
    S.set_al_state(5.0, 5.0)
    g = torch.empty(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    view = S.assemble_hessian(T(x), g)
    Hg, lam_g, _ = gpu_hessian(S, view)
    m, y, ps = oracle_state(sc, x, 5.0)
    g_or = system.gradient(m, x, y, ps, 5.0).ravel()
    H_or, lam_or = system.hessian(m, x, y, ps, 5.0, with_lambda=True)
    gerr = np.abs(g.cpu().numpy() - g_or).max() / np.abs(g_or).max()
    D = (Hg - H_or).toarray()
    herr = np.abs(D).max() / np.abs(H_or.toarray()).max()
    lerr = np.abs(lam_g - lam_or).max() / np.abs(lam_or).max()
    assert gerr < 1e-10, gerr
    assert herr < HESS_TOL_F32, herr
    assert herr > 1e-12, herr            # the FP32 kernel did run (FP64 would agree to ~1e-15)
    assert lerr < HESS_TOL_F32, lerr
    assert np.abs(D - D.T).max() <= 1e-12 * np.abs(H_or.toarray()).max()   # symmetric storage


def test_fp32_time_step_matches_oracle():
    sc = close_cubes(n=2, gap=5e-4)
    S = bal.Scene(sc, bal.default_params(newton_tol=1e-8, pcg_tol=1e-10, precision=bal.PREC_FP32,
                                         mixed_max_refine=40))
    m = system.make_model(sc)
    compare_trajectory(S, m, sc, 2, obal.Params(newton_tol=1e-8), T)


def test_fp32_solve_reports_its_precision():
    sc = close_cubes(n=2)
    S = bal.Scene(sc, bal.default_params(precision=bal.PREC_FP32))
    S.step_begin(T(sc.X), T(sc.V0))
    g = torch.empty(3 * sc.n_verts, dtype=torch.float64, device=DEV)
    S.assemble_hessian(T(sc.X), g)
    sol = torch.zeros_like(g)
    info = S.pcg_solve(-g, sol, 1e-8, 5000)
    assert info["precision_used"] == bal.PREC_FP32
    assert info["rel_residual"] <= 1e-8
