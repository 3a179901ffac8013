"""FP32 + FP64-refinement PCG with the difference form of the FP32 operator
on a stiff system, against the oracle.

The system is the first Newton system (x = x_t, no contact) of a 3 x 3 piece
of the interlocked chain net: 21 torus links of E = 1 GPa, the eight border
rings pinned, so the free links carry near-rigid modes whose eigenvalues of
D^-1 H are m_v / h^2 over the stiff diagonal -- the kappa that defeats FP32.
Rounding every block of H to FP32 (the plain form) moves those modes by
eps_32 |D| |v|; the difference form, (H v)_i = G_i v_i + sum_j B_ij (v_j - v_i)
with G_i summed in FP64 before rounding, moves them by eps_32 |B| |v_j - v_i|
only -- translations exactly not at all -- because every stencil Hessian
except the mass term is translation invariant (Sec. 3.1 objective: elastic
energy and contact distances depend on position differences).

Checked: the difference form converges to the FP64 relative residual 1e-6 and
its solution solves the ORACLE's assembled system (FP64, CPU) to that
tolerance; the plain form, given the same inner caps and passes, either does
not converge or needs more FP32 iterations."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import system  # noqa: E402
from paper_2407_00046_b300 import bal, scenes  # noqa: E402

TOL = 1e-6
MAX_IT = 60000
FORM_PARAMS = dict(precision=bal.PREC_MIXED, pcg_stall_window=20000, mixed_inner_max=2000,
                   mixed_inner_tol=1e-2, mixed_max_refine=40)


@pytest.fixture(scope="module")
def stiff_net():
    sc = scenes.chain_net_shells(nx=3, nz=3, n_shells=0, link_theta=24, link_cross=2)
    model = system.make_model(sc)
    y = system.inertia_target(model, sc.X, sc.V0)
    ps = system.empty_pairs()
    H = system.hessian(model, sc.X, y, ps, 0.0)
    e = system.gradient(model, sc.X, y, ps, 0.0).ravel()
    S = bal.Scene(sc, bal.default_params(**FORM_PARAMS))
    x0 = torch.tensor(sc.X, dtype=torch.float64, device="cuda").contiguous()
    v0 = torch.tensor(sc.V0, dtype=torch.float64, device="cuda").contiguous()
    S.step_begin(x0, v0)
    g = torch.empty_like(x0)
    view = S.assemble_hessian(x0, g)
    assert view["nnz_C"] == 0
    return S, g.view(-1), H, e


def _solve(S, g, op):
    S.set_params(mixed_operator=op, **FORM_PARAMS)
    sol = torch.zeros_like(g)
    info = S.pcg_solve(-g, sol, TOL, MAX_IT)
    return sol.cpu().numpy(), info


def test_difference_form_converges_on_stiff_links(stiff_net):
    S, g, H, e = stiff_net
    p, info = _solve(S, g, bal.MIXED_OP_DIFFERENCE)
    b = -e
    res = float(np.linalg.norm(b - H @ p) / np.linalg.norm(b))
    print(f"\n[difference] iters {info['iters']} passes {info['refine_passes']} "
          f"converged {info['converged']} oracle residual {res:.3e}")
    assert info["converged"] == 1 and info["refine_passes"] >= 1
    assert res <= 1.05 * TOL, res


def test_plain_form_needs_more_or_fails(stiff_net):
    S, g, H, e = stiff_net
    p_d, info_d = _solve(S, g, bal.MIXED_OP_DIFFERENCE)
    p_p, info_p = _solve(S, g, bal.MIXED_OP_PLAIN)
    b = -e
    res_p = float(np.linalg.norm(b - H @ p_p) / np.linalg.norm(b))
    print(f"\n[plain] iters {info_p['iters']} passes {info_p['refine_passes']} converged "
          f"{info_p['converged']} oracle residual {res_p:.3e}; [difference] iters {info_d['iters']}")
    assert info_d["converged"] == 1
    assert (not info_p["converged"]) or info_p["iters"] > info_d["iters"]
    # a pass that raises the FP64 residual is rolled back: never worse than x = 0
    assert res_p <= 1.0 + 1e-12
