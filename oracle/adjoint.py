"""FP64 adjoint of the BAL time step (not in the paper; test infrastructure).

At a converged step, grad_x L(x_{t+1}; x_t, v_t, E) = 0 with the final AL
state (A at x_{t+1}, A', mu, s, sigma) held fixed. Differentiating:
H lambda = a, H = unprojected Hessian of L at x_{t+1},
a = dJ/dx_{t+1} + dJ/dv_{t+1} / h (because v_{t+1} = (x_{t+1} - x_t)/h), and
y = x_t + h v_t + h^2 g enters grad L as M (x - y) / h^2, so on free vertices
    dJ/dx_t = M lambda / h^2 - dJ/dv_{t+1} / h,   dJ/dv_t = M lambda / h,
and, with mu, lam linear in E, d(grad W_e)/dE_e = grad W_e / E_e:
    dJ/dE_e = -lambda_e^T grad W_e / E_e.
"""
import numpy as np

from . import bal, elastic, system


def forward(model, x0, v0, steps, prm, frozen=None):
    """Rollout with checkpoints (x_t, v_t, x_{t+1}, sigma, A' -> mu). With
    frozen = [(sigma, A' -> mu)] per step, each step is solved with that AL
    state held fixed (the map the adjoint differentiates)."""
    x, v = np.array(x0, dtype=np.float64), np.array(v0, dtype=np.float64)
    ckpt = []
    for k in range(steps):
        xt, vt = x.copy(), v.copy()
        x, v, info = bal.time_step(model, x, v, prm, frozen=None if frozen is None else frozen[k])
        if not info["converged"]:
            raise RuntimeError("oracle step did not converge")
        ckpt.append((xt, vt, x.copy(), info["sigma"], dict(info["Ap"])))
    return x, v, ckpt


def step_adjoint(model, xt, vt, xn, sigma, Ap, gx, gv):
    """dJ/dx_t, dJ/dv_t and dJ/dE for one step."""
    sc = model.scene
    h = model.h
    y = system.inertia_target(model, xt, vt)
    keys, _ = bal.active_pairs(model, xn)
    ps = bal.make_pairset(model, xn, keys, Ap, sigma)
    H = system.hessian(model, xn, y, ps, sigma, project=False)
    a = (gx + gv / h).copy()
    a[~model.free] = 0.0
    lam = bal.solve(H, a.ravel()).reshape(-1, 3)
    m = model.mass[:, None]
    dx = m * lam / h ** 2 - gv / h
    dv = m * lam / h
    dx[~model.free] = 0.0
    dv[~model.free] = 0.0
    _, g_el, _ = elastic.element_terms(xn, sc.tets, model.Dm_inv, model.vol, model.mu, model.lam,
                                       project=False)
    lam_e = lam[sc.tets].reshape(-1, 12)
    dE = -np.sum(lam_e * g_el, axis=1) / np.asarray(sc.E)
    return dx, dv, dE


def backward(model, ckpt, gx, gv):
    dE = np.zeros(model.scene.n_tets)
    for xt, vt, xn, sigma, Ap in reversed(ckpt):
        gx, gv, de = step_adjoint(model, xt, vt, xn, sigma, Ap, gx, gv)
        dE += de
    return gx, gv, dE
