"""torch.autograd.Function over T time steps of libbal (the adjoint is not in
the paper): forward runs bal_time_step and keeps a checkpoint per step
(x_t, v_t, x_{t+1}, converged AL state); backward replays the checkpoints in
reverse through bal_adjoint_step, which solves H lambda = dL/dx_{t+1} +
dL/dv_{t+1}/h with the unprojected Hessian at x_{t+1} and returns the
gradients with respect to x_t, v_t and per-tet Young's modulus E."""
import torch

from . import bal as _bal


class _Simulate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, E, v0, x0, scene, steps, adj_tol, require_converged=True, stats=None, checkpoints=None):
        scene.set_materials(E.detach().cpu().double().numpy())
        x = x0.detach().clone().contiguous()
        v = v0.detach().clone().contiguous()
        ckpt = []
        ctx.unconverged = 0
        for _ in range(steps):
            xt, vt = x.clone(), v.clone()
            info = scene.time_step(x, v, check=False)
            if not info["converged"]:
                if require_converged:
                    raise _bal.BalError(3, "time step did not converge in the differentiated run")
                ctx.unconverged += 1   # the adjoint of that step is then approximate
            ckpt.append((xt, vt, x.clone(), scene.get_al_state()))
        ctx.scene, ctx.ckpt, ctx.nt, ctx.adj_tol = scene, ckpt, E.numel(), adj_tol
        if stats is not None:
            stats.append({"steps": steps, "unconverged_steps": ctx.unconverged})
        if checkpoints is not None:
            checkpoints.extend(ckpt)
        ctx.infos = []
        return x.clone(), v.clone()

    @staticmethod
    def backward(ctx, gx, gv):
        S = ctx.scene
        ref = ctx.ckpt[0][0]
        gx = torch.zeros_like(ref) if gx is None else gx.detach().double().contiguous()
        gv = torch.zeros_like(ref) if gv is None else gv.detach().double().contiguous()
        dE = torch.zeros(ctx.nt, dtype=torch.float64, device=ref.device)
        for xt, vt, xn, al in reversed(ctx.ckpt):
            gx, gv, info = S.adjoint_step(xt, vt, xn, al, gx, gv, dE, rel_tol=ctx.adj_tol)
            ctx.infos.append(info)
        return dE, gv, gx, None, None, None, None, None, None


def simulate(scene, x0, v0, E, steps, adj_tol=1e-12, require_converged=True, stats=None, checkpoints=None):
    """Differentiable T-step rollout: returns (x_T, v_T); gradients flow to
    E [n_tets], v0 and x0 [n_verts*3] (CUDA float64 tensors). With
    require_converged=False a step that ends at the Newton cap is kept and its
    adjoint is that of an approximate minimiser; stats (a list) receives the
    number of such steps; checkpoints (a list) receives the per-step
    checkpoints (x_t, v_t, x_{t+1}, AL state)."""
    return _Simulate.apply(E, v0, x0, scene, steps, adj_tol, require_converged, stats, checkpoints)
