"""Benchmark of the BAL inexact Newton-PCG path on one B300.

Workload (default): the heterogeneous net scene -- an interlocked torus-link
chain net (E = 1 GPa, border links pinned) under four spiked spherical shells
(E = 5e5 Pa) dropped from 2 cm, ~1.77M tets, h = 1/30 s, dhat = 1e-3 m,
synthetic and seeded (it stands in for the paper's "Puffer Balls on Nets",
Table 1).

First --time-steps whole time steps are run from the initial state to
convergence of Algorithm 1, each timed with CUDA events (the ms-per-time-step
half of the metric; reported under "time_steps"). Then the benchmark steps:
W warm-up and K timed Algorithm 1 iterations of the following time step(s),
each one pass of the whole hot path (contact detection, projected-Hessian
assembly, PCG solve, step bound and line search, AL update). value = PCG
iterations per second over the K timed iterations (all ranks); ms_per_step =
ms per Algorithm 1 iteration. The matrix is larger than L2 at this size, so no
L2 flush is inserted. `--impl reference` times the FP64 CPU oracle on a bounded
sample instead. Multi-GPU: independent replicas of the scene, one per rank
(weak scaling; the path has no collective).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG iters/s and ms per time step at 1.7M tets; BSR SpMV % of HBM peak"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        except Exception:
            return out
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = float(rows[0][2])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = set()
        for r in rows:
            if len(r) < 9:
                continue
            for k, name in enumerate(names):
                if r[5 + k].strip() == "Active":
                    seen.add(name)
        out["reasons"] = sorted(seen)
        out["samples"] = len(rows)
        return out


# FP64 instructions per tet of k_elastic_hess<double> (projected Hessian: F,
# signed SVD by 3x3 Jacobi, the analytic eigensystem of the 9x9 dP/dF, the
# 12x12 block and its slot scatter), from the ncu SASS counters of one launch
# on the 1,771,008-tet chain net (profiles/k_elastic_hess_chain_net_shells.md):
# DADD 0.30 G, DMUL 0.84 G, DFMA 1.75 G. DADD and DMUL occupy the FP64 pipe
# like DFMA, so the pipe's ceiling is the FMA issue rate (measured FP64 FMA
# TFLOP/s / 2); flops count DFMA twice.
ELASTIC_HESS_DADD_PER_TET = 0.30e9 / 1771008
ELASTIC_HESS_DMUL_PER_TET = 0.84e9 / 1771008
ELASTIC_HESS_DFMA_PER_TET = 1.75e9 / 1771008


PRECISIONS = {"fp64": 0, "mixed": 1, "df64": 2, "fp32": 3}     # bal_precision values
PRECONDS = {"block-jacobi": 0, "warm-start": 1, "additive": 2}   # bal_precond values
STEP_MODES = {"ca": 0, "ccd": 1}                     # bal_step_mode values
BROAD_PHASES = {"grid": 0, "lbvh": 1}                # bal_broad_phase values
AL_MODES = {"algorithm1": 0, "plain": 1}             # bal_al_mode values
PCG_TOL_MODES = {"fixed": 0, "truncated-newton": 1, "cond-x": 2, "cond-b": 3}  # bal_pcg_tol_mode values
DTYPES = {"fp64": "f64", "mixed": "f32+f64", "df64": "df64+f64", "fp32": "f32+f64"}


def spmv_kernel_bytes(precision, nv, nnzL, nnzC):
    """Name and algorithmic bytes of one timed SpMV of a PCG iteration.

    df64 (k_dd_spmv): the method-minimal symmetric storage (Sec. 5.1) read
    once -- diagonal and lower blocks as 8-byte double-floats, one column index
    per block, the row pointer -- plus one read of p and one write of q. The
    column-side index lists and the second (L2) read of each block for its
    transpose are this kernel's overhead, not algorithmic.
    fp64 / mixed / fp32 (k_pcg_offdiag): lower blocks with their row and column index,
    one read of p, q read and written once."""
    nb = nnzL + nnzC
    if precision == "df64":
        return ("k_dd_spmv (symmetric H p, double-float gather)",
                (nv + nb) * 72 + nb * 4 + (nv + 1) * 4 + 2 * 24 * nv)
    p = 4 if precision in ("mixed", "fp32") else 8
    return "k_pcg_offdiag (symmetric off-diagonal blocks, atomics)", nb * (9 * p + 8) + 3 * 3 * nv * p


def pcg_iteration_bytes(nv, nnzL, nnzC):
    """Method-minimal bytes of one block-Jacobi PCG iteration with 8-byte
    values (FP64 or double-float): the symmetric SpMV (matrix read once, p
    read, q written) plus the vector work fused into two passes -- x += alpha p,
    r -= alpha q, z = D^-1 r (read x, p, q, r and D^-1; write x, r, z) and
    p = z + beta p (read z, p; write p): 24 B per vertex per vector access,
    72 B per D^-1 block, 312 B per vertex in all."""
    _, spmv = spmv_kernel_bytes("df64", nv, nnzL, nnzC)
    return spmv + (7 * 24 + 72 + 3 * 24) * nv


def pcg_iteration_roofline(precision, nv, nnzL, nnzC, iters_per_s, peak, peak_kind):
    """The whole PCG iteration against the measured HBM bandwidth: its
    method-minimal bytes at the PCG-only iteration rate (8-byte-value forms)."""
    if precision not in ("df64", "fp64") or not iters_per_s:
        return None
    byts = pcg_iteration_bytes(nv, nnzL, nnzC)
    gbs = byts * iters_per_s / 1e9
    return {"bound": "hbm", "unit": "GB/s", "bytes_per_iteration": byts, "iters_per_s": round(iters_per_s, 1),
            "achieved": round(gbs, 1), "peak": peak, "peak_kind": peak_kind, "frac": round(gbs / peak, 4),
            "note": "SpMV, update and direction kernels of one iteration; the rate is pcg_only_iters_per_s"}


# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture on the chain-net workload (profiles/k_dd_spmv_chain_net_shells.md),
# valid while the kernel's sources hash to the values recorded with it.
NCU_TRAFFIC = {
    ("df64", "chain_net_shells"): {
        "bytes": 267.28e6,     # mean of two launches: 259.3 + 9.7 and 258.6 + 6.9 MB
        "sources": {"paper_2407_00046_b300/csrc/ddpcg.cu": "5a38744b69c14847",
                    "paper_2407_00046_b300/csrc/dd.cuh": "bdb727145b83135d"},
    },
}


def ncu_traffic(precision, scene):
    import hashlib
    rec = NCU_TRAFFIC.get((precision, scene))
    if rec is None:
        return None
    root = os.path.dirname(os.path.abspath(__file__))
    for path, want in rec["sources"].items():
        with open(os.path.join(root, path), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != want:
                return None   # the kernel changed since the counters were taken
    return rec["bytes"]


def roofline_entry(precision, kname, achieved, peak, peak_kind, byts, ms, n, nv, nnzL, nnzC, traffic=None,
                   fp64_peak=None):
    out = {"kernel": kname, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
           "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
           "traffic": traffic, "bytes_per_launch": byts, "ms_per_launch": round(ms, 5),
           "timed_launches": n, "nnz_L": nnzL, "nnz_C_last": nnzC}
    if precision == "fp64" and fp64_peak:
        flops = 36.0 * (nnzL + nnzC)
        tf = flops / (ms * 1e-3) / 1e12
        out["alu"] = {"bound": "alu", "unit": "FP64 TFLOP/s", "achieved": round(tf, 4),
                      "peak": round(fp64_peak, 4), "frac": round(tf / fp64_peak, 4),
                      "peak_kind": "measured in this run (bal_fp64_fma_rate)"}
    return out


def assembly_bytes(n_tets, nv, nnzL, n_pairs):
    """Algorithmic bytes of one assembly: per tet its 4 indices, D_m^-1 (9 f64)
    and V, mu, lambda; positions read once; the diagonal and static lower
    blocks written once (f64); per contact pair its key and 10 emitted
    blocks (4 diagonal, 6 off-diagonal) written and read once by the merge."""
    return n_tets * (16 + 72 + 24) + nv * 24 + (nv + nnzL) * 72 + n_pairs * (8 + 2 * 10 * 72)


def assembly_roofline(n_tets, nv, nnzL, n_pairs, elastic_ms, total_ms, n, fp64_peak, hbm_peak, peak_kind):
    """The element Hessian kernel against the measured FP64 FMA rate (it is
    bound by the FP64 pipe on B300), and the whole assembly's algorithmic
    bytes against the measured HBM copy bandwidth."""
    if n == 0:
        return None
    e_ms, t_ms = elastic_ms / n, total_ms / n
    instr = (ELASTIC_HESS_DADD_PER_TET + ELASTIC_HESS_DMUL_PER_TET + ELASTIC_HESS_DFMA_PER_TET) * n_tets
    flop = (ELASTIC_HESS_DADD_PER_TET + ELASTIC_HESS_DMUL_PER_TET + 2 * ELASTIC_HESS_DFMA_PER_TET) * n_tets
    ti = instr / (e_ms * 1e-3) / 1e12
    ipeak = fp64_peak / 2.0
    byts = assembly_bytes(n_tets, nv, nnzL, n_pairs)
    gbs = byts / (t_ms * 1e-3) / 1e9
    return {"kernel": "k_elastic_hess<double>", "bound": "alu", "unit": "T FP64 instr/s",
            "achieved": round(ti, 4), "peak": round(ipeak, 4), "frac": round(ti / ipeak, 4),
            "peak_kind": "measured in this run (bal_fp64_fma_rate / 2: one FP64 pipe instruction per FMA)",
            "flop_tflops": round(flop / (e_ms * 1e-3) / 1e12, 4), "ms_per_launch": round(e_ms, 4),
            "fp64_instr_per_tet": round(instr / n_tets, 1), "timed_assemblies": n,
            "hbm": {"what": "whole assembly (element + contact stencils, duplicate merge, D^-1)",
                    "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(gbs / hbm_peak, 4), "peak_kind": peak_kind, "bytes": byts,
                    "ms_per_assembly": round(t_ms, 4), "contact_pairs_last": n_pairs}}


def run_pcg_only(args):
    """Assemble the Hessian of the workload once (at x_0 + one gravity step, the
    free-fall iterate) and run a fixed number of PCG iterations on it: the
    SpMV / PCG kernels in isolation (used for profiling)."""
    import torch
    from paper_2407_00046_b300 import bal, build, scenes
    build.build(force=False, verbose=False)
    dev = torch.device("cuda", 0)
    sc = scenes.scene_by_name(args.scene)
    params = bal.default_params(pcg_stall_window=1 << 30,
                                precision=PRECISIONS[args.precision],
                                broad_phase=BROAD_PHASES[args.broad_phase],
                                mixed_inner_max=args.pcg_iters, mixed_max_refine=1, mixed_inner_tol=0.0,
                                spmv_window=args.spmv_window)
    S = bal.Scene(sc, params, pair_capacity=args.pair_capacity)
    x = torch.tensor(sc.X, dtype=torch.float64, device=dev)
    v = torch.tensor(sc.V0, dtype=torch.float64, device=dev)
    warm_steps = getattr(args, "pcg_warm_steps", 0)
    if warm_steps > 0:
        # reach a state in contact first: time steps with the bench's solver settings
        S.set_params(_scene_params(args, bal))
        for _ in range(warm_steps):
            S.time_step(x, v, check=False)
        S.set_params(params)
    S.step_begin(x, v)
    g = torch.empty_like(x)
    view = S.assemble_hessian(x, g)
    b = -g
    sol = torch.zeros_like(b)
    S.pcg_solve(b, sol, 0.0, 20)
    times = []
    S.kernel_timing(True)
    for _ in range(max(args.steps, 1)):
        sol.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        info = S.pcg_solve(b, sol, 0.0, args.pcg_iters)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / max(info["iters"], 1))
    k_ms, k_n = S.kernel_timing(False)
    ms = statistics.median(times)
    kname, byts = spmv_kernel_bytes(args.precision, sc.n_verts, view["nnz_L"], view["nnz_C"])
    kms = k_ms / max(k_n, 1)
    return {"mode": "pcg", "scene": args.scene, "precision": args.precision,
            "iters_per_solve": args.pcg_iters, "ms_per_iter": round(ms, 4),
            "iters_per_s": round(1e3 / ms, 1), "nnz_L": view["nnz_L"], "nnz_C": view["nnz_C"],
            "warm_steps": warm_steps, "n_verts": sc.n_verts,
            "spmv_kernel": kname, "spmv_ms_per_launch": round(kms, 5),
            "spmv_gbs": round(byts / (kms * 1e-3) / 1e9, 1), "spmv_bytes": byts,
            "pcg_iteration_bytes": pcg_iteration_bytes(sc.n_verts, view["nnz_L"], view["nnz_C"]),
            "pcg_iteration_gbs": round(pcg_iteration_bytes(sc.n_verts, view["nnz_L"], view["nnz_C"])
                                       / (ms * 1e-3) / 1e9, 1)}


def _scene_params(args, bal, **kw):
    return bal.default_params(pcg_tol=args.pcg_tol, newton_tol=args.newton_tol,
                              newton_max_iter=args.newton_max, pcg_stall_window=args.pcg_stall,
                              pcg_max_iter=args.pcg_max, precision=PRECISIONS[args.precision],
                              precond=PRECONDS[args.precond], step_mode=STEP_MODES[args.step_mode],
                              broad_phase=BROAD_PHASES[args.broad_phase], spmv_window=args.spmv_window,
                              pcg_stall_forcing=args.pcg_stall_forcing, **kw)


def run_adjoint(args):
    """Gradient of a loss after --adj-steps steps (the squared distance of the
    first body's centroid to the scene's target) with respect to per-tet E and
    the initial velocity, through the autograd.Function: forward (time steps
    with a checkpoint each) and backward (one adjoint solve per step) timed
    separately. Default scene: the 105k-tet cube dropped on the 202k-tet slab."""
    import torch
    from paper_2407_00046_b300 import bal, build, scenes
    from paper_2407_00046_b300.autograd import simulate
    build.build(force=False, verbose=False)
    dev = torch.device("cuda", 0)
    name = args.scene if args.scene != "chain_net_shells" else "cube_on_slab"
    sc = scenes.scene_by_name(name)
    S = bal.Scene(sc, _scene_params(args, bal), pair_capacity=1 << 22)
    mass = torch.tensor(S.mass(), device=dev)
    body = torch.tensor(np.flatnonzero(sc.body == 0), device=dev)
    target = torch.tensor(sc.info.get("target", sc.X.mean(0)), dtype=torch.float64, device=dev)
    E = torch.tensor(sc.E, dtype=torch.float64, device=dev, requires_grad=True)
    v0 = torch.tensor(sc.V0, dtype=torch.float64, device=dev).view(-1).requires_grad_(True)
    x0 = torch.tensor(sc.X, dtype=torch.float64, device=dev).view(-1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    stats, ckpts = [], []
    xT, vT = simulate(S, x0, v0, E, args.adj_steps, require_converged=False, stats=stats, checkpoints=ckpts)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    m = mass[body]
    c = (m[:, None] * xT.view(-1, 3)[body]).sum(0) / m.sum()
    J = ((c - target) ** 2).sum()
    J.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    out = {"mode": "adjoint", "scene": name, "n_tets": sc.n_tets, "n_verts": sc.n_verts,
           "steps": args.adj_steps, "precision_forward": args.precision,
           "forward_ms_per_step": round(1e3 * (t1 - t0) / args.adj_steps, 1),
           "backward_ms_per_step": round(1e3 * (t2 - t1) / args.adj_steps, 1),
           "unconverged_forward_steps": stats[0]["unconverged_steps"] if stats else None,
           "newton_cap": args.newton_max, "newton_tol": args.newton_tol,
           "loss": float(J.detach()), "grad_E_norm": float(E.grad.norm()), "grad_v0_norm": float(v0.grad.norm()),
           "data": "synthetic (seeded procedural scene)"}
    if args.adj_fd:
        out["fd_check"] = adjoint_fd_check(S, x0, E, v0, mass, body, target, [c[3] for c in ckpts], args)
    return out


def adjoint_fd_check(S, x0, E, v0, mass, body, target, frozen, args, h=1e-6):
    """Central finite differences of the same --adj-steps rollout, each step
    re-solved with the AL state (sigma, A', mu) its differentiated run ended
    with (the map the adjoint differentiates): along one random direction of
    the per-tet E (relative step h) and one of the cube's initial velocity
    (h m/s), and along --adj-fd-entries single entries of each with the
    largest adjoint gradients. Reports adjoint and FD values and their
    relative differences."""
    import torch
    rng = np.random.default_rng(17)
    dev = x0.device
    gE = E.grad.detach().clone()
    gv = v0.grad.detach().clone()
    E0 = E.detach().clone()

    def rollout(Evals, vinit):
        S.set_materials(Evals.cpu().numpy())
        x, v = x0.clone(), vinit.clone()
        S.set_params(freeze_al=1)
        for f in frozen:
            S.set_al_state(f["sigma"], f["sigma0"], f["ap_keys"], f["ap_mu"])
            S.time_step(x, v, check=False)
        S.set_params(freeze_al=0)
        m = mass[body]
        c = (m[:, None] * x.view(-1, 3)[body]).sum(0) / m.sum()
        return float(((c - target) ** 2).sum())

    checks = []

    def fd(name, dE_rel, dv, adj):
        t0 = time.perf_counter()
        jp = rollout(E0 * (1 + h * dE_rel), v0.detach() + h * dv)
        jm = rollout(E0 * (1 - h * dE_rel), v0.detach() - h * dv)
        val = (jp - jm) / (2 * h)
        print(f"[bench] fd {name}: adjoint {adj:.9e} fd {val:.9e} ({time.perf_counter() - t0:.0f} s)",
              file=sys.stderr, flush=True)
        checks.append({"what": name, "adjoint": adj, "fd": val,
                       "rel_diff": abs(adj - val) / max(abs(val), 1e-300)})

    zE = torch.zeros_like(E0)
    zv = torch.zeros_like(gv)
    w = torch.tensor(rng.choice([-1.0, 1.0], size=E0.numel()), dtype=torch.float64, device=dev)
    fd("E random direction (relative)", w, zv, float((gE * E0 * w).sum()))
    u = torch.zeros_like(gv).view(-1, 3)
    u[body] = torch.tensor(rng.normal(size=(body.numel(), 3)), dtype=torch.float64, device=dev)
    u = u.view(-1)
    fd("v0 random direction", zE, u, float((gv * u).sum()))
    for i in torch.argsort((gE * E0).abs(), descending=True)[:args.adj_fd_entries].tolist():
        e = zE.clone()
        e[i] = 1.0
        fd(f"E[{i}] (relative)", e, zv, float(gE[i] * E0[i]))
    for i in torch.argsort(gv.abs(), descending=True)[:args.adj_fd_entries].tolist():
        e = zv.clone()
        e[i] = 1.0
        fd(f"v0[{i}]", zE, e, float(gv[i]))
    S.set_materials(E0.cpu().numpy())
    return {"h": h, "checks": checks, "max_rel_diff": max(c["rel_diff"] for c in checks)}


def run_precision_sweep(args):
    """The same --steps time steps from the scene's initial state in each
    solver precision: ms per step, Newton and PCG iterations, and the largest
    vertex distance to the FP64 run. Default scene: the 1.05M-tet stack of 64
    cubes with E log-uniform in [1e5, 1e9]."""
    import torch
    from paper_2407_00046_b300 import bal, build, scenes
    build.build(force=False, verbose=False)
    dev = torch.device("cuda", 0)
    name = args.scene if args.scene != "chain_net_shells" else "cube_columns"
    sc = scenes.scene_by_name(name)
    out, ref = {}, None
    for prec in ("fp64", "df64", "mixed"):
        a = argparse.Namespace(**vars(args))
        a.precision = prec
        S = bal.Scene(sc, _scene_params(a, bal, mixed_inner_max=3000, mixed_max_refine=60,
                                        mixed_inner_tol=1e-2), pair_capacity=1 << 22)
        x = torch.tensor(sc.X, dtype=torch.float64, device=dev).contiguous()
        v = torch.tensor(sc.V0, dtype=torch.float64, device=dev).contiguous()
        infos = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(max(args.steps, 1)):
            infos.append(S.time_step(x, v, check=False))
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        xs = x.cpu().numpy()
        if ref is None:
            ref = xs
        out[prec] = {"ms_per_step": round(1e3 * sec / max(args.steps, 1), 1),
                     "newton_iters": [i["newton_iters"] for i in infos],
                     "pcg_iters": [i["pcg_iters_total"] for i in infos],
                     "converged": [i["converged"] for i in infos],
                     "max_vertex_diff_vs_fp64_m": float(np.abs(xs - ref).max())}
        del S
    return {"mode": "precision-sweep", "scene": name, "n_tets": sc.n_tets, "n_verts": sc.n_verts,
            "steps": args.steps, "pcg_tol": args.pcg_tol, "results": out,
            "data": "synthetic (seeded procedural scene)"}


def budgeted_time_step(S, x, v, stream, budget_s):
    """One time step through the public calls -- bal_step_begin, Algorithm 1
    iterations (bal_newton_step) until the convergence test, the Newton cap or
    the wall-clock budget, bal_step_end -- with the bal_time_step summary."""
    t0 = time.perf_counter()
    S.step_begin(x, v, stream=stream)
    out = {"newton_iters": 0, "pcg_iters_total": 0, "converged": 0, "max_active": 0,
           "min_distance": float("inf"), "ms_assemble": 0.0, "ms_solve": 0.0, "ms_line_search": 0.0,
           "ms_contact": 0.0, "status": 3, "budget_hit": 0}       # 3: BAL_ERR_NOT_CONVERGED
    out["sigma0"] = S.get_al_state()["sigma0"]
    for _ in range(S.get_params().newton_max_iter):
        ni = S.newton_step(x, stream=stream, check=False)
        for kk in ("ms_assemble", "ms_solve", "ms_line_search", "ms_contact"):
            out[kk] += ni[kk]
        out["pcg_iters_total"] += ni["pcg_iters"]
        out["max_active"] = max(out["max_active"], ni["n_active"])
        out["min_distance"] = min(out["min_distance"], ni["dmin"])
        if ni["status"] != 0:
            out["status"] = ni["status"]
            break
        if ni["converged"]:
            out["status"], out["converged"] = 0, 1
            break
        out["newton_iters"] += 1
        if time.perf_counter() - t0 > budget_s:
            out["budget_hit"] = 1
            break
    out["sigma_final"] = S.get_al_state()["sigma"]
    S.step_end(x, v, stream=stream)
    return out


def reduce_over_ranks(ms, e2e_ms, pcg_iters, e2e_iters, world, dev=None):
    """Whole-job figures of a replicas-only run: the slowest rank's times (max)
    and the PCG iterations of all ranks (sum). One collective per figure kind,
    outside the timed region; identity for a single process."""
    if world <= 1:
        return ms, e2e_ms, pcg_iters, e2e_iters
    import torch
    t = torch.tensor([ms, e2e_ms, float(pcg_iters), float(e2e_iters)], dtype=torch.float64, device=dev)
    mx = t.clone()
    torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
    sm = t.clone()
    torch.distributed.all_reduce(sm, op=torch.distributed.ReduceOp.SUM)
    return float(mx[0]), float(mx[1]), float(sm[2]), float(sm[3])


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_ours(args, rank, world):
    """Time steps of the workload to convergence from its initial state (each
    one timed with CUDA events: the ms-per-time-step half of the metric), then
    the benchmark proper: W warm-up and K timed Algorithm 1 iterations of the
    following time step(s) in contact. One bench step = one Algorithm 1
    iteration = one pass of the whole hot path (contact detection, assembly of
    the projected Hessian, PCG solve, step bound and line search, AL update);
    when a time step converges inside the run the next one begins (v update,
    new inertia target and sigma0) and the iterations continue."""
    import torch
    from paper_2407_00046_b300 import bal, build, scenes

    build.build(force=False, verbose=False)
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    sc = scenes.scene_by_name(args.scene)
    params = _scene_params(args, bal, warm_tol=args.warm_tol, warm_max_iter=args.warm_iters,
                           al_mode=AL_MODES[args.al_mode], pcg_tol_mode=PCG_TOL_MODES[args.pcg_tol_mode],
                           friction=args.friction, sigma_literal_max=int(args.sigma_rule == "printed"))
    S = bal.Scene(sc, params, pair_capacity=1 << 22)
    stream = torch.cuda.current_stream()
    x = torch.tensor(sc.X, dtype=torch.float64, device=dev).contiguous()
    v = torch.tensor(sc.V0, dtype=torch.float64, device=dev).contiguous()

    def progress(tag, info, ms):
        print(f"[bench] {tag}: status {info['status']} newton {info['newton_iters']} pcg "
              f"{info['pcg_iters_total']} max|A| {info['max_active']} min d {info['min_distance']:.3e} "
              f"sigma {info['sigma_final']:.4g} ms {ms:.0f} (asm {info['ms_assemble']:.0f} solve "
              f"{info['ms_solve']:.0f} ls {info['ms_line_search']:.0f} contact {info['ms_contact']:.0f})",
              file=sys.stderr, flush=True)

    # 1. whole time steps to convergence (Newton cap --newton-max), one by one,
    # within a wall-clock budget for the phase (a step still open when it runs
    # out ends unconverged, like one at the Newton cap, and no further step starts)
    time_steps = []
    t_phase = time.perf_counter()
    for k in range(args.time_steps):
        left = args.time_step_budget - (time.perf_counter() - t_phase)
        if left <= 0:
            break
        e0, e1 = _events()
        e0.record(stream)
        info = budgeted_time_step(S, x, v, stream, left)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        progress(f"time step {k}", info, ms)
        time_steps.append({"step": k, "status": info["status"], "converged": int(info["converged"]),
                           "ms": round(ms, 1), "newton_iters": info["newton_iters"],
                           "pcg_iters": info["pcg_iters_total"], "max_active": info["max_active"],
                           "min_distance": info["min_distance"], "sigma0": info["sigma0"],
                           "sigma_final": info["sigma_final"], "budget_hit": info["budget_hit"],
                           "phase_ms": {kk: round(info[kk], 1) for kk in
                                        ("ms_assemble", "ms_solve", "ms_line_search", "ms_contact")}})

    # 2. Algorithm 1 iterations of the next time step(s)
    S.step_begin(x, v, stream=stream)
    state = {"time_steps_done": 0}

    def alg1_iteration(xx):
        ni = S.newton_step(xx, stream=stream, check=False)
        if ni["status"] not in (0, 7):       # OK, or a line search below alpha_min (reported)
            raise RuntimeError(f"Algorithm 1 iteration failed: status {ni['status']}: {bal.last_error()}")
        if ni["converged"]:                  # the time step is over: start the next one
            S.step_end(xx, v, stream=stream)
            S.step_begin(xx, v, stream=stream)
            state["time_steps_done"] += 1
        return ni

    for _ in range(args.warmup):
        alg1_iteration(x)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = _events()
    timed = []
    launches0 = bal.launch_count()
    S.kernel_timing(True)
    with Clocks(dev.index) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            timed.append(alg1_iteration(x))
        e1.record(stream)
        torch.cuda.synchronize()
    launches = bal.launch_count() - launches0
    k_ms, k_n = S.kernel_timing(False)
    a_el_ms, a_tot_ms, a_n = S.assembly_timing()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    pcg_iters = sum(t["pcg_iters"] for t in timed)

    # end to end through the public API with host buffers: every iteration
    # copies its input positions from pinned host memory and its result back
    xh = x.cpu().pin_memory()
    torch.cuda.synchronize()
    f0, f1 = _events()
    f0.record(stream)
    e2e_iters = 0
    for _ in range(args.steps):
        x.copy_(xh, non_blocking=True)
        e2e_iters += alg1_iteration(x)["pcg_iters"]
        xh.copy_(x, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1)

    # roofline of the dominant kernel: the SpMV of every PCG iteration, timed
    # per launch with CUDA events on the solve stream during the timed region
    view = S.assemble_hessian(x)
    nv, nnzL, nnzC = sc.n_verts, view["nnz_L"], view["nnz_C"]
    kname, byts = spmv_kernel_bytes(args.precision, nv, nnzL, nnzC)
    spmv_ms = k_ms / max(k_n, 1)
    peak, peak_kind = peaks()
    achieved = byts / (spmv_ms * 1e-3) / 1e9
    fp64_peak = bal.fp64_fma_rate(stream=stream)
    max_pairs = max((t["n_active"] for t in timed), default=0)
    # PCG-only iteration rate on the same system (fixed iteration count)
    rhs = torch.randn(3 * nv, dtype=torch.float64, device=dev)
    sol = torch.zeros_like(rhs)
    keep = S.get_params()
    S.set_params(pcg_stall_window=1 << 30)
    S.pcg_solve(rhs, sol, 0.0, 10)
    sol.zero_()
    torch.cuda.synchronize()
    p0 = time.perf_counter()
    pi = S.pcg_solve(rhs, sol, 0.0, 200)
    torch.cuda.synchronize()
    pcg_only = pi["iters"] / (time.perf_counter() - p0)
    S.set_params(keep)
    forms = precision_forms(S, sc, dev, args) if not args.no_forms else None

    ms, e2e_ms, pcg_iters, e2e_iters = reduce_over_ranks(ms, e2e_ms, pcg_iters, e2e_iters, world, dev)
    if rank != 0:
        return None
    value = pcg_iters / (ms * 1e-3)
    e2e_val = e2e_iters / (e2e_ms * 1e-3)
    contact_steps = [t for t in time_steps if t["max_active"] > 0]
    conv_contact = [t for t in contact_steps if t["converged"]]
    line = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "PCG iter/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": DTYPES[args.precision],
        "data": "synthetic (seeded procedural scene, no paper meshes)",
        "config": {
            "workload": f"{sc.name}: {sc.n_tets} tets, {sc.n_verts} verts, h=1/30 s, dhat=1e-3 m",
            "step": "one Algorithm 1 iteration (contact detection, projected-Hessian assembly, PCG, "
                    "step bound + line search, AL update) of the time steps that follow the "
                    "converged ones below",
            "scene": args.scene, "n_tets": sc.n_tets, "n_verts": sc.n_verts,
            "pcg_tol": args.pcg_tol, "pcg_max_iter": args.pcg_max, "newton_tol": args.newton_tol,
            "pcg_stall_window": args.pcg_stall, "newton_cap": args.newton_max,
            "spmv_window": args.spmv_window, "pcg_stall_forcing": args.pcg_stall_forcing,
            "sigma_rule": args.sigma_rule,
            "precond": args.precond, "precision": args.precision,
            "step_bound": args.step_mode, "broad_phase": args.broad_phase,
            "al_mode": args.al_mode, "pcg_tol_mode": args.pcg_tol_mode,
            "friction": args.friction,
            "l2": "no flush: Hessian storage exceeds the 126 MB L2",
            "parallelism": f"replicas x{world}",
        },
        "time_steps": {
            "ms_per_time_step": (round(statistics.mean(t["ms"] for t in conv_contact), 1)
                                 if conv_contact else None),
            "newton_iters_per_time_step": (round(statistics.mean(t["newton_iters"] for t in conv_contact), 1)
                                           if conv_contact else None),
            "contact_steps_converged": f"{len(conv_contact)}/{len(contact_steps)}",
            "converged": f"{sum(t['converged'] for t in time_steps)}/{len(time_steps)}",
            "capped_ms": [t["ms"] for t in contact_steps if not t["converged"]],
            "note": "each time step from the initial state run to convergence (Alg. 1 test "
                    "||e||/||e0|| <= newton_tol), the Newton cap or the phase's wall-clock "
                    "budget (budget_hit), timed with CUDA events; ms_per_time_step and "
                    "newton_iters_per_time_step are the means over the steps in contact that "
                    "converged (null if none did); capped_ms lists the contact steps that "
                    "did not converge",
            "budget_s": args.time_step_budget,
            "steps": time_steps,
        },
        "alg1_iterations": {
            "pcg_iters_per_iteration": round(pcg_iters / max(args.steps, 1) / max(world, 1), 1),
            "max_active_pairs": max((t["n_active"] for t in timed), default=0),
            "min_distance": min((t["dmin"] for t in timed), default=None),
            "pcg_rel_residual_max": max((t["pcg_rel_residual"] for t in timed if t["pcg_iters"] > 0),
                                        default=None),
            "pcg_iters_per_solve": [t["pcg_iters"] for t in timed],
            "time_steps_completed_in_run": state["time_steps_done"],
            "phase_ms_per_iteration": {k: round(sum(t[k] for t in timed) / max(args.steps, 1), 2)
                                       for k in ("ms_assemble", "ms_solve", "ms_line_search", "ms_contact")},
        },
        "max_active_pairs": max([t["max_active"] for t in time_steps] + [t["n_active"] for t in timed]),
        "pcg_only_iters_per_s": round(pcg_only, 1),
        "roofline_pcg_iteration": pcg_iteration_roofline(args.precision, nv, nnzL, nnzC, pcg_only, peak,
                                                         peak_kind),
        "e2e": {"value": round(e2e_val, 2), "unit": "PCG iter/s",
                "h2d_bytes_per_step": 3 * nv * 8, "d2h_bytes_per_step": 3 * nv * 8},
        "roofline": roofline_entry(args.precision, kname, achieved, peak, peak_kind, byts, spmv_ms,
                                   k_n, nv, nnzL, nnzC, ncu_traffic(args.precision, args.scene), fp64_peak),
        "roofline_assembly": assembly_roofline(sc.n_tets, nv, nnzL, max_pairs, a_el_ms, a_tot_ms, a_n,
                                               fp64_peak, peak, peak_kind),
        "fp64_fma_tflops": round(fp64_peak, 4),
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if forms is not None:
        line["precision_forms"] = forms
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, nv, nnzL, nnzC)
    return line


# The forms are compared on one system solved to the tolerance, so the
# stagnation window must not end the 11k-iteration block-Jacobi solves of the
# 1 GPa net early (the time-step bench uses a shorter one).
FORMS_STALL_WINDOW = 20000
# FP32 + refinement restarts CG every pass and its FP32 operator differs from
# H by ~kappa eps_32 on the stiff modes, so it takes several times the FP64
# form's iterations on the net.
FORMS_MAX_ITER_MIXED = 100000


def precision_forms(S, sc, dev, args):
    """The solver forms -- three precisions with block-Jacobi (the FP32 +
    FP64-refinement form with the FP32 operator in difference form, inner caps
    of 3k and 10k FP32 iterations per pass, and in the plain form), and in FP64
    the additive (App. A) and warm-start (Sec. 4.2.2) preconditioners -- on the
    same system: the first Newton system of the workload's first step (x =
    x_0, no contact; the 1 GPa links make it the stiff part, kappa ~ 1e8) --
    solved from zero to the bench tolerance: iterations, time, FP64 relative
    residual and the relative difference of the solution to the FP64 one."""
    import torch
    from paper_2407_00046_b300 import bal
    keep = S.get_params()
    x0 = torch.tensor(sc.X, dtype=torch.float64, device=dev).contiguous()
    v0 = torch.tensor(sc.V0, dtype=torch.float64, device=dev).contiguous()
    S.step_begin(x0, v0)
    g = torch.empty_like(x0)
    S.assemble_hessian(x0, g)
    b = -g.view(-1)
    out, ref = {}, None
    # (name, precision, preconditioner, FP32 inner iteration cap, FP32 operator form)
    diff, plain = bal.MIXED_OP_DIFFERENCE, bal.MIXED_OP_PLAIN
    forms = [("fp64", "fp64", "block-jacobi", 0, diff), ("df64", "df64", "block-jacobi", 0, diff),
             ("mixed", "mixed", "block-jacobi", 3000, diff),
             ("mixed_inner10k", "mixed", "block-jacobi", 10000, diff),
             ("mixed_plain", "mixed", "block-jacobi", 3000, plain),
             ("fp64_additive", "fp64", "additive", 0, diff), ("fp64_warm_start", "fp64", "warm-start", 0, diff)]
    for name, prec, pc, inner, op in forms:
        S.set_params(precision=PRECISIONS[prec], precond=PRECONDS[pc], pcg_stall_window=FORMS_STALL_WINDOW,
                     mixed_inner_max=max(inner, 1), mixed_max_refine=60, mixed_inner_tol=1e-2,
                     mixed_operator=op, warm_tol=args.warm_tol, warm_max_iter=args.warm_iters)
        sol = torch.zeros_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            info = S.pcg_solve(b, sol, args.pcg_tol, FORMS_MAX_ITER_MIXED if prec == "mixed" else 30000)
        except bal.BalError as e:          # reported, not fatal to the line
            out[name] = {"error": str(e)}
            continue
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        if ref is None:
            ref = sol.clone()
        diff_rel = float((sol - ref).abs().max() / ref.abs().max().clamp_min(1e-300))
        out[name] = {"iters": info["iters"], "seconds": round(sec, 3), "converged": info["converged"],
                     "rel_residual": info["rel_residual"], "refine_passes": info["refine_passes"],
                     "max_rel_diff_vs_fp64": diff_rel, "precision_used": info["precision_used"],
                     "warm_iters": info["warm_iters"]}
        if prec == "mixed":
            out[name]["fp32_operator"] = "difference" if op == diff else "plain"
    S.set_params(keep)
    out["system"] = "first Newton system of step 1 (x = x_0), rhs = -gradient, x from 0"
    return out


def run_forms(args):
    """--mode forms: only the solver-form comparison (precision_forms) on the
    workload's first Newton system."""
    import torch
    from paper_2407_00046_b300 import bal, build, scenes
    build.build(force=False, verbose=False)
    dev = torch.device("cuda", 0)
    sc = scenes.scene_by_name(args.scene)
    S = bal.Scene(sc, _scene_params(args, bal), pair_capacity=1 << 22)
    out = precision_forms(S, sc, dev, args)
    return {"mode": "forms", "scene": args.scene, "n_tets": sc.n_tets, "n_verts": sc.n_verts,
            "pcg_tol": args.pcg_tol, "forms": out, "data": "synthetic (seeded procedural scene)"}


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or None


def cpu_baseline(args, nv_full, nnzL_full, nnzC_full, budget_s=15.0):
    """The FP64 oracle timed on this host's cores on a bounded sample: oracle
    assembly of a small chain-net scene and scipy CSR matvec of its Hessian,
    scaled by stored blocks to one PCG iteration (SpMV + 3 vector passes) of the
    full workload. The matvec runs on one thread ("cores"); the host's core
    count and CPU model are recorded beside it."""
    from oracle import system
    from paper_2407_00046_b300 import scenes
    t0 = time.perf_counter()
    sc = scenes.scene_by_name("chain_net_shells_small")
    m = system.make_model(sc)
    y = system.inertia_target(m, sc.X, sc.V0)
    ta = time.perf_counter()
    H = system.hessian(m, sc.X, y, system.empty_pairs(), 1.0)
    t_asm = time.perf_counter() - ta
    v = np.random.default_rng(0).normal(size=H.shape[0])
    reps, tm = 0, time.perf_counter()
    while time.perf_counter() - tm < min(5.0, budget_s):
        H @ v
        reps += 1
    t_spmv = (time.perf_counter() - tm) / reps
    stored_small = H.nnz
    stored_full = 9 * (nv_full + 2 * (nnzL_full + nnzC_full))
    w = np.random.default_rng(1).normal(size=3 * nv_full)
    tv = time.perf_counter()
    for _ in range(3):
        w = w + 0.5 * w
        float(w @ w)
    t_vec = time.perf_counter() - tv
    t_iter = t_spmv * stored_full / stored_small + t_vec
    return {"value": round(1.0 / t_iter, 3), "unit": "PCG iter/s", "cores": 1, "kind": "oracle",
            "host_cores": os.cpu_count(), "cpu_model": _cpu_model(),
            "sample": (f"oracle assembly ({sc.n_tets} tets, {t_asm:.2f} s) and scipy CSR matvec "
                       f"({stored_small} stored entries, {t_spmv * 1e3:.2f} ms) of a 3x3-ring "
                       f"chain net with one shell, scaled to {stored_full} stored entries "
                       f"+ 3 vector passes of the full scene; single thread"),
            "seconds": round(time.perf_counter() - t0, 1)}


def run_reference(args):
    t0 = time.perf_counter()
    from paper_2407_00046_b300 import scenes
    sc = scenes.scene_by_name(args.scene)
    # stored blocks of the full workload from its static pattern (contact part
    # not included: the reference arm has no GPU assembly to report it)
    pairs = set()
    T = sc.tets.astype(np.int64)
    for a in range(4):
        for b in range(a + 1, 4):
            lo, hi = np.minimum(T[:, a], T[:, b]), np.maximum(T[:, a], T[:, b])
            pairs.update((hi * sc.n_verts + lo).tolist())
    nnzL = len(pairs)
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(args, sc.n_verts, nnzL, 0, budget_s=2.0)
    for _ in range(args.steps):
        vals.append(cpu_baseline(args, sc.n_verts, nnzL, 0, budget_s=5.0))
    ms = (time.perf_counter() - t0) * 1e3
    value = statistics.median(v["value"] for v in vals)
    return {
        "metric": METRIC, "value": value, "unit": "PCG iter/s", "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / max(args.steps, 1), 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": f"{sc.name}: {sc.n_tets} tets", "scene": args.scene},
        "cpu_baseline": vals[-1],
        "e2e": {"value": value, "unit": "PCG iter/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10,
                    help="timed bench steps: Algorithm 1 iterations (one pass of the hot path each)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--time-step-budget", type=float, default=540.0,
                    help="wall-clock seconds for the --time-steps phase (keeps the default run bounded)")
    ap.add_argument("--time-steps", type=int, default=3,
                    help="time steps run to convergence and timed one by one before the bench steps "
                         "(free fall, impact, first step in contact on the default workload)")
    ap.add_argument("--sigma-rule", default="printed", choices=["printed", "capped"],
                    help="Alg. 1 sigma update: the printed max(1.2 sigma, 100 sigma0), or the capped "
                         "reading min(1.2 sigma, 100 sigma0)")
    ap.add_argument("--pcg-max", type=int, default=10000, help="PCG iteration cap per solve")
    ap.add_argument("--pcg-stall-forcing", type=float, default=0.5,
                    help="eta > 0: the stagnation window may end a PCG solve only once ||r|| <= eta ||r0||")
    ap.add_argument("--spmv-window", type=int, default=0,
                    help="double-float SpMV: 0 = row gather with full column-side lists; W = windows "
                         "of W rows with in-window transposes summed in shared memory")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scene", default="chain_net_shells")
    ap.add_argument("--precision", default="df64", choices=sorted(PRECISIONS))
    ap.add_argument("--pcg-tol", type=float, default=1e-6)
    ap.add_argument("--newton-tol", type=float, default=1e-4)
    ap.add_argument("--newton-max", type=int, default=2000,
                    help="Algorithm 1 iterations per time step (cap; the step reports convergence); "
                         "the --time-steps phase is bounded by --time-step-budget as well")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the three-precision comparison")
    ap.add_argument("--precond", default="block-jacobi", choices=sorted(PRECONDS),
                    help="block-Jacobi PCG, or preceded by the stiffness-grouped warm start (Sec. 4.2.2)")
    ap.add_argument("--step-mode", default="ccd", choices=sorted(STEP_MODES),
                    help="line-search step bound: conservative advancement or cubic CCD (Sec. 5.3)")
    ap.add_argument("--broad-phase", default="lbvh", choices=sorted(BROAD_PHASES))
    ap.add_argument("--al-mode", default="algorithm1", choices=sorted(AL_MODES),
                    help="Algorithm 1, or the plain inexact Newton ablation (sigma = sigma0, no A')")
    ap.add_argument("--pcg-tol-mode", default="fixed", choices=sorted(PCG_TOL_MODES),
                    help="fixed --pcg-tol, or App. B criterion (i) min(0.5, sqrt(||e||))")
    ap.add_argument("--friction", type=float, default=0.0,
                    help="friction coefficient chi of the fully-implicit friction (0 = frictionless)")
    ap.add_argument("--warm-tol", type=float, default=1e-2)
    ap.add_argument("--warm-iters", type=int, default=50)
    ap.add_argument("--pcg-stall", type=int, default=2000,
                    help="PCG stagnation window (App. B uses 100; at 100 the block-Jacobi solves of "
                         "the 1 GPa net stop before their residual starts to fall)")
    ap.add_argument("--mode", default="step", choices=["step", "pcg", "adjoint", "precision-sweep", "forms"],
                    help="pcg: assemble once and time fixed-length PCG solves (profiling); adjoint: "
                         "forward + backward of --adj-steps steps through the autograd.Function; "
                         "precision-sweep: the same steps in FP64, df64 and FP32 + refinement; forms: "
                         "only the solver-form comparison on the first Newton system")
    ap.add_argument("--adj-steps", type=int, default=20)
    ap.add_argument("--adj-fd", action="store_true",
                    help="--mode adjoint: central FD check of the gradient (AL state frozen per step)")
    ap.add_argument("--adj-fd-entries", type=int, default=0,
                    help="--adj-fd: also this many single E and v0 entries (largest gradients)")
    ap.add_argument("--pcg-iters", type=int, default=200)
    ap.add_argument("--pair-capacity", type=int, default=1 << 22,
                    help="--mode pcg: contact pair capacity of the scene (device memory for contact buffers)")
    ap.add_argument("--pcg-warm-steps", type=int, default=0,
                    help="--mode pcg: time steps taken before the assembly (a state in contact)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.mode in ("pcg", "adjoint", "precision-sweep", "forms"):
        run = {"pcg": run_pcg_only, "adjoint": run_adjoint, "precision-sweep": run_precision_sweep,
               "forms": run_forms}
        if rank == 0:
            print(json.dumps(run[args.mode](args)), flush=True)
        return
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
