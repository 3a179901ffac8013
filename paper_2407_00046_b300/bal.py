"""Thin Python binding of libbal (ctypes): argument marshalling only.

Every numerical step runs in the CUDA kernels of libbal.so; this module only
turns torch CUDA tensors into device pointers and the C structs into dicts.
It fails loudly if the library is missing or was built without a GPU
present -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbal.so")

OK = 0
STATUS = {0: "OK", 1: "ARG", 2: "CAPACITY", 3: "NOT_CONVERGED", 4: "NAN", 5: "TIMEOUT",
          6: "CUDA", 7: "LINE_SEARCH", 8: "STATE"}
PREC_FP64, PREC_MIXED, PREC_DF64, PREC_FP32 = 0, 1, 2, 3
MIXED_OP_DIFFERENCE, MIXED_OP_PLAIN = 0, 1   # bal_mixed_operator values
PRECOND_BJ, PRECOND_BJ_WARMSTART, PRECOND_ADDITIVE = 0, 1, 2
STEP_CA, STEP_CCD = 0, 1
BROAD_GRID, BROAD_LBVH = 0, 1
AL_ALGORITHM1, AL_PLAIN = 0, 1
PCG_TOL_FIXED, PCG_TOL_TRUNCATED_NEWTON, PCG_TOL_COND_X, PCG_TOL_COND_B = 0, 1, 2, 3


class BalError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libbal {STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("precision", C.c_int32), ("precond", C.c_int32), ("pcg_tol", C.c_double),
                ("pcg_max_iter", C.c_int32), ("pcg_stall_window", C.c_int32),
                ("newton_tol", C.c_double), ("newton_abs_tol", C.c_double),
                ("newton_max_iter", C.c_int32), ("ap_ratio", C.c_double),
                ("sigma_growth", C.c_double), ("sigma_cap", C.c_double),
                ("sigma_literal_max", C.c_int32), ("step_bound", C.c_double),
                ("ls_min_alpha", C.c_double), ("ls_slack", C.c_double),
                ("contact_cap", C.c_int64), ("ls_extra_pcg", C.c_int32),
                ("warm_tol", C.c_double), ("warm_max_iter", C.c_int32),
                ("mixed_inner_max", C.c_int32), ("mixed_inner_tol", C.c_double),
                ("mixed_max_refine", C.c_int32), ("ca_max_iter", C.c_int32),
                ("freeze_al", C.c_int32), ("step_mode", C.c_int32), ("broad_phase", C.c_int32),
                ("al_mode", C.c_int32), ("pcg_tol_mode", C.c_int32),
                ("friction", C.c_double), ("friction_eps_v", C.c_double),
                ("spmv_window", C.c_int32), ("ls_extra_rounds", C.c_int32),
                ("pcg_stall_forcing", C.c_double), ("mixed_operator", C.c_int32)]


class SceneDesc(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tets", C.c_int32), ("n_tris", C.c_int32),
                ("n_edges", C.c_int32), ("n_surf_verts", C.c_int32),
                ("X", C.c_void_p), ("tets", C.c_void_p), ("tris", C.c_void_p),
                ("edges", C.c_void_p), ("surf_verts", C.c_void_p), ("E", C.c_void_p),
                ("nu", C.c_void_p), ("rho", C.c_void_p), ("pinned", C.c_void_p),
                ("h", C.c_double), ("dhat", C.c_double), ("gravity", C.c_double * 3),
                ("pair_capacity", C.c_int64), ("pair_limit", C.c_int64)]


class BsrView(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("nnz_L", C.c_int64), ("nnz_C", C.c_int64),
                ("D", C.c_void_p), ("L_row_ptr", C.c_void_p), ("L_col", C.c_void_p),
                ("L_val", C.c_void_p), ("C_row", C.c_void_p), ("C_col", C.c_void_p),
                ("C_val", C.c_void_p), ("Lambda", C.c_void_p)]


class ALState(C.Structure):
    _fields_ = [("sigma", C.c_double), ("sigma0", C.c_double), ("dmin_prev", C.c_double),
                ("n_ap", C.c_int64), ("ap_keys", C.c_void_p), ("ap_mu", C.c_void_p)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("rel_residual", C.c_double),
                ("rel_residual_r0", C.c_double), ("stagnated", C.c_int32),
                ("converged", C.c_int32), ("refine_passes", C.c_int32),
                ("warm_iters", C.c_int32), ("n_groups", C.c_int32),
                ("negative_curvature", C.c_int32), ("precision_used", C.c_int32)]


class NewtonInfo(C.Structure):
    _fields_ = [("l", C.c_int32), ("converged", C.c_int32), ("n_active", C.c_int64),
                ("n_ap", C.c_int64), ("n_candidates", C.c_int64), ("dmin", C.c_double),
                ("sigma", C.c_double), ("grad_norm", C.c_double), ("alpha", C.c_double),
                ("ls_trials", C.c_int32), ("pcg_iters", C.c_int32),
                ("pcg_rel_residual", C.c_double), ("energy", C.c_double),
                ("ms_assemble", C.c_double), ("ms_solve", C.c_double),
                ("ms_line_search", C.c_double), ("ms_contact", C.c_double),
                ("ms_ls_broad", C.c_double), ("ms_ls_bound", C.c_double),
                ("ms_ls_energy", C.c_double), ("n_raw_candidates", C.c_int64),
                ("pcg_tol", C.c_double), ("kappa", C.c_double)]


class StepInfo(C.Structure):
    _fields_ = [("newton_iters", C.c_int32), ("pcg_iters_total", C.c_int32),
                ("converged", C.c_int32), ("max_active", C.c_int64),
                ("min_distance", C.c_double), ("sigma0", C.c_double),
                ("sigma_final", C.c_double), ("ms_total", C.c_double),
                ("ms_assemble", C.c_double), ("ms_solve", C.c_double),
                ("ms_line_search", C.c_double), ("ms_contact", C.c_double)]


def _as_dict(s):
    return {f: getattr(s, f) for f, _ in s._fields_}


_LIB = None
P = C.c_void_p


def load(path: str = LIB_PATH):
    """Loads libbal.so (raises if it is missing: no fallback exists)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} not built; run python -m paper_2407_00046_b300.build")
    lib = C.CDLL(path)
    sigs = {
        "bal_last_error": ([], C.c_char_p),
        "bal_launch_count": ([], C.c_uint64),
        "bal_struct_size": ([C.c_int32], C.c_uint64),
        "bal_default_params": ([C.POINTER(Params)], None),
        "bal_create_scene": ([C.POINTER(SceneDesc), C.POINTER(Params), C.POINTER(P)], C.c_int),
        "bal_destroy_scene": ([P], C.c_int),
        "bal_set_params": ([P, C.POINTER(Params)], C.c_int),
        "bal_get_params": ([P, C.POINTER(Params)], C.c_int),
        "bal_kernel_timing": ([P, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64)], C.c_int),
        "bal_fp64_fma_rate": ([C.c_int32, C.POINTER(C.c_double), P], C.c_int),
        "bal_assembly_timing": ([P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int64)],
                                C.c_int),
        "bal_step_bound": ([P, P, P, P, C.c_int64, C.c_int32, C.POINTER(C.c_double), P], C.c_int),
        "bal_find_candidates": ([P, P, P, C.c_double, P, C.c_int64, C.POINTER(C.c_int64), P], C.c_int),
        "bal_static_pattern": ([P, C.POINTER(C.c_int64), P, P], C.c_int),
        "bal_get_mass": ([P, P], C.c_int),
        "bal_step_begin": ([P, P, P, P], C.c_int),
        "bal_step_end": ([P, P, P, P], C.c_int),
        "bal_get_al_state": ([P, C.POINTER(ALState), C.c_int64], C.c_int),
        "bal_set_al_state": ([P, C.POINTER(ALState)], C.c_int),
        "bal_get_y": ([P, P, P], C.c_int),
        "bal_assemble_hessian": ([P, P, P, C.POINTER(BsrView), P], C.c_int),
        "bal_copy_hessian": ([P, P, P, P, P, P, P, P], C.c_int),
        "bal_spmv": ([P, P, P, P], C.c_int),
        "bal_pcg_solve": ([P, P, P, C.c_double, C.c_int32, C.POINTER(SolveInfo), P], C.c_int),
        "bal_energy": ([P, P, C.POINTER(C.c_double), P], C.c_int),
        "bal_newton_step": ([P, P, C.POINTER(NewtonInfo), P], C.c_int),
        "bal_time_step": ([P, P, P, C.POINTER(StepInfo), P], C.c_int),
        "bal_set_materials": ([P, P, P], C.c_int),
        "bal_adjoint_step": ([P, P, P, P, C.POINTER(ALState), P, P, P, P, P, C.c_double, C.c_int32,
                              C.POINTER(SolveInfo), P], C.c_int),
        "bal_pcg_solve_noalloc": ([C.c_int32, P, C.c_int64, P, P, P, P, P, C.c_double, C.c_int32,
                                   C.POINTER(SolveInfo), P], C.c_int),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = lib
    return lib


def _check(status):
    if status != OK:
        raise BalError(status, load().bal_last_error().decode())


def fp64_fma_rate(iters: int = 20000, stream=None) -> float:
    """Measured FP64 FMA throughput of the current device, TFLOP/s."""
    t = C.c_double()
    _check(load().bal_fp64_fma_rate(int(iters), C.byref(t), _stream(stream)))
    return t.value


def last_error() -> str:
    """The library's message for the last failed call on this thread."""
    return load().bal_last_error().decode()


def launch_count() -> int:
    """Kernels launched by libbal in this process so far."""
    return int(load().bal_launch_count())


def default_params(**kw) -> Params:
    p = Params()
    load().bal_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _dev(t, dtype=None, numel=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Scene:
    """A libbal scene built from a paper_2407_00046_b300.scenes.Scene."""

    def __init__(self, scene, params: Params | None = None, pair_capacity: int = 1 << 16,
                 pair_limit: int = (1 << 31) - 1):
        lib = load()
        self.src = scene
        self.nv = scene.n_verts
        self._keep = dict(
            X=np.ascontiguousarray(scene.X, dtype=np.float64),
            tets=np.ascontiguousarray(scene.tets, dtype=np.int32),
            tris=np.ascontiguousarray(scene.tris, dtype=np.int32),
            edges=np.ascontiguousarray(scene.edges, dtype=np.int32),
            surf=np.ascontiguousarray(scene.surf_verts, dtype=np.int32),
            E=np.ascontiguousarray(scene.E, dtype=np.float64),
            nu=np.ascontiguousarray(scene.nu, dtype=np.float64),
            rho=np.ascontiguousarray(scene.rho, dtype=np.float64),
            pinned=np.ascontiguousarray(scene.pinned, dtype=np.uint8))
        k = self._keep
        d = SceneDesc()
        d.n_verts, d.n_tets = scene.n_verts, scene.n_tets
        d.n_tris, d.n_edges, d.n_surf_verts = len(k["tris"]), len(k["edges"]), len(k["surf"])
        for name, key in (("X", "X"), ("tets", "tets"), ("tris", "tris"), ("edges", "edges"),
                          ("surf_verts", "surf"), ("E", "E"), ("nu", "nu"), ("rho", "rho"),
                          ("pinned", "pinned")):
            setattr(d, name, k[key].ctypes.data)
        d.h, d.dhat = float(scene.h), float(scene.dhat)
        for i in range(3):
            d.gravity[i] = float(scene.gravity[i])
        d.pair_capacity, d.pair_limit = pair_capacity, pair_limit
        self.params = params if params is not None else default_params()
        self._h = C.c_void_p()
        _check(lib.bal_create_scene(C.byref(d), C.byref(self.params), C.byref(self._h)))

    def close(self):
        if self._h:
            load().bal_destroy_scene(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- parameters / static data ------------------------------------------------
    def set_params(self, params: Params | None = None, **kw):
        p = params if params is not None else self.get_params()
        for k, v in kw.items():
            setattr(p, k, v)
        _check(load().bal_set_params(self._h, C.byref(p)))
        self.params = p

    def kernel_timing(self, enable: bool):
        """(total ms, launches) of the timed SpMV kernel of each PCG iteration
        since the previous call; resets them and switches timing on or off."""
        ms, n = C.c_double(), C.c_int64()
        _check(load().bal_kernel_timing(self._h, int(bool(enable)), C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def assembly_timing(self):
        """(element-kernel ms, whole-assembly ms, assemblies) since the last call."""
        e, t, n = C.c_double(), C.c_double(), C.c_int64()
        _check(load().bal_assembly_timing(self._h, C.byref(e), C.byref(t), C.byref(n)))
        return e.value, t.value, n.value

    def get_params(self) -> Params:
        p = Params()
        _check(load().bal_get_params(self._h, C.byref(p)))
        return p

    def static_pattern(self):
        nnz = C.c_int64()
        _check(load().bal_static_pattern(self._h, C.byref(nnz), None, None))
        rp = np.zeros(self.nv + 1, np.int32)
        col = np.zeros(max(nnz.value, 1), np.int32)
        _check(load().bal_static_pattern(self._h, C.byref(nnz), rp.ctypes.data_as(P),
                                         col.ctypes.data_as(P)))
        return rp, col[:nnz.value]

    def mass(self):
        m = np.zeros(self.nv)
        _check(load().bal_get_mass(self._h, m.ctypes.data_as(P)))
        return m

    # ---- time step state -------------------------------------------------------------
    def step_begin(self, x_t, v_t, stream=None):
        import torch
        n = 3 * self.nv
        _check(load().bal_step_begin(self._h, _dev(x_t, torch.float64, n), _dev(v_t, torch.float64, n),
                                     _stream(stream)))

    def step_end(self, x, v_out, stream=None):
        """v_out = (x - x_t) / h for the step begun by step_begin (device)."""
        import torch
        n = 3 * self.nv
        _check(load().bal_step_end(self._h, _dev(x, torch.float64, n), _dev(v_out, torch.float64, n),
                                   _stream(stream)))

    def get_al_state(self):
        st = ALState()
        _check(load().bal_get_al_state(self._h, C.byref(st), 0))
        n = st.n_ap
        keys = np.zeros(max(n, 1), np.uint64)
        mu = np.zeros(max(n, 1))
        st.ap_keys, st.ap_mu = keys.ctypes.data, mu.ctypes.data
        _check(load().bal_get_al_state(self._h, C.byref(st), n))
        return dict(sigma=st.sigma, sigma0=st.sigma0, dmin_prev=st.dmin_prev,
                    ap_keys=keys[:n].copy(), ap_mu=mu[:n].copy())

    def set_al_state(self, sigma, sigma0, ap_keys=(), ap_mu=(), dmin_prev=float("inf")):
        keys = np.ascontiguousarray(np.asarray(ap_keys, dtype=np.uint64))
        mu = np.ascontiguousarray(np.asarray(ap_mu, dtype=np.float64))
        st = ALState(sigma, sigma0, dmin_prev, len(keys), keys.ctypes.data if len(keys) else None,
                     mu.ctypes.data if len(mu) else None)
        _check(load().bal_set_al_state(self._h, C.byref(st)))

    def get_y(self, out, stream=None):
        import torch
        _check(load().bal_get_y(self._h, _dev(out, torch.float64, 3 * self.nv), _stream(stream)))
        return out

    # ---- hot path ------------------------------------------------------------------------
    def assemble_hessian(self, x, grad_out=None, stream=None):
        import torch
        v = BsrView()
        g = _dev(grad_out, torch.float64, 3 * self.nv) if grad_out is not None else None
        _check(load().bal_assemble_hessian(self._h, _dev(x, torch.float64, 3 * self.nv), g,
                                           C.byref(v), _stream(stream)))
        return _as_dict(v)

    def copy_hessian(self, view, stream=None):
        """Device copies of the assembled blocks: dict of torch tensors."""
        import torch
        dev = torch.device("cuda")
        out = dict(D=torch.empty(self.nv * 9, dtype=torch.float64, device=dev),
                   L=torch.empty(max(view["nnz_L"], 1) * 9, dtype=torch.float64, device=dev),
                   C_row=torch.empty(max(view["nnz_C"], 1), dtype=torch.int32, device=dev),
                   C_col=torch.empty(max(view["nnz_C"], 1), dtype=torch.int32, device=dev),
                   C_val=torch.empty(max(view["nnz_C"], 1) * 9, dtype=torch.float64, device=dev),
                   Lambda=torch.empty(self.nv * 3, dtype=torch.float64, device=dev))
        _check(load().bal_copy_hessian(self._h, _dev(out["D"]), _dev(out["L"]), _dev(out["C_row"]),
                                       _dev(out["C_col"]), _dev(out["C_val"]), _dev(out["Lambda"]),
                                       _stream(stream)))
        out["L"] = out["L"][:view["nnz_L"] * 9]
        for k in ("C_row", "C_col"):
            out[k] = out[k][:view["nnz_C"]]
        out["C_val"] = out["C_val"][:view["nnz_C"] * 9]
        return out

    def spmv(self, v, y, stream=None):
        import torch
        n = 3 * self.nv
        _check(load().bal_spmv(self._h, _dev(v, torch.float64, n), _dev(y, torch.float64, n),
                               _stream(stream)))
        return y

    def pcg_solve(self, rhs, sol, rel_tol, max_iter, stream=None):
        import torch
        n = 3 * self.nv
        info = SolveInfo()
        _check(load().bal_pcg_solve(self._h, _dev(rhs, torch.float64, n), _dev(sol, torch.float64, n),
                                    float(rel_tol), int(max_iter), C.byref(info), _stream(stream)))
        return _as_dict(info)

    def energy(self, x, stream=None):
        import torch
        e = C.c_double()
        _check(load().bal_energy(self._h, _dev(x, torch.float64, 3 * self.nv), C.byref(e),
                                 _stream(stream)))
        return e.value

    def find_candidates(self, x, r, direction=None, capacity=1 << 22, stream=None):
        """Broad-phase candidate pair keys (sorted int64 device tensor) at x, or
        swept along direction."""
        import torch
        n3 = 3 * self.nv
        out = torch.empty(capacity, dtype=torch.int64, device="cuda")
        n = C.c_int64()
        d = _dev(direction, torch.float64, n3) if direction is not None else None
        _check(load().bal_find_candidates(self._h, _dev(x, torch.float64, n3), d, float(r),
                                          C.c_void_p(out.data_ptr()), int(capacity), C.byref(n),
                                          _stream(stream)))
        return out[:n.value].clone()

    def step_bound(self, x, direction, keys, mode, stream=None):
        """Line-search step bound over the pair keys (uint64 device tensor or
        host sequence) along x + t direction: mode STEP_CA or STEP_CCD."""
        import torch
        n = 3 * self.nv
        k = keys if isinstance(keys, torch.Tensor) else torch.tensor(
            [int(v) for v in keys], dtype=torch.int64)
        k = k.to(device="cuda", dtype=torch.int64).contiguous()
        a = C.c_double()
        _check(load().bal_step_bound(self._h, _dev(x, torch.float64, n), _dev(direction, torch.float64, n),
                                     C.c_void_p(k.data_ptr()), int(k.numel()), int(mode), C.byref(a),
                                     _stream(stream)))
        return a.value

    def newton_step(self, x, stream=None, check=True):
        import torch
        info = NewtonInfo()
        s = load().bal_newton_step(self._h, _dev(x, torch.float64, 3 * self.nv), C.byref(info),
                                   _stream(stream))
        if check:
            _check(s)
        d = _as_dict(info)
        d["status"] = s
        return d

    def set_materials(self, E, nu=None):
        """Per-tet Young's modulus (and Poisson ratio) from host arrays."""
        E = np.ascontiguousarray(np.asarray(E, dtype=np.float64))
        nu = np.ascontiguousarray(np.asarray(self._keep["nu"] if nu is None else nu, dtype=np.float64))
        _check(load().bal_set_materials(self._h, E.ctypes.data_as(P), nu.ctypes.data_as(P)))
        self._keep["E"], self._keep["nu"] = E, nu

    def adjoint_step(self, x_t, v_t, x_next, al, dLdx_next, dLdv_next, dLdE_accum,
                     rel_tol=1e-12, max_iter=100000, stream=None):
        """One step of the adjoint: returns (dL/dx_t, dL/dv_t, info); adds into dLdE_accum."""
        import torch
        n = 3 * self.nv
        keys = np.ascontiguousarray(np.asarray(al["ap_keys"], dtype=np.uint64))
        mu = np.ascontiguousarray(np.asarray(al["ap_mu"], dtype=np.float64))
        st = ALState(al["sigma"], al["sigma0"], al.get("dmin_prev", float("inf")), len(keys),
                     keys.ctypes.data if len(keys) else None, mu.ctypes.data if len(mu) else None)
        dx = torch.empty_like(dLdx_next)
        dv = torch.empty_like(dLdv_next)
        info = SolveInfo()
        _check(load().bal_adjoint_step(
            self._h, _dev(x_t, torch.float64, n), _dev(v_t, torch.float64, n),
            _dev(x_next, torch.float64, n), C.byref(st), _dev(dLdx_next, torch.float64, n),
            _dev(dLdv_next, torch.float64, n), _dev(dx, torch.float64, n), _dev(dv, torch.float64, n),
            _dev(dLdE_accum, torch.float64, self.src.n_tets), float(rel_tol), int(max_iter),
            C.byref(info), _stream(stream)))
        return dx, dv, _as_dict(info)

    def time_step(self, x, v, stream=None, check=True):
        import torch
        info = StepInfo()
        n = 3 * self.nv
        s = load().bal_time_step(self._h, _dev(x, torch.float64, n), _dev(v, torch.float64, n),
                                 C.byref(info), _stream(stream))
        if check:
            _check(s)
        d = _as_dict(info)
        d["status"] = s
        return d


NOALLOC_MAX_VERTS = 16384


def pcg_solve_noalloc(D, rows, cols, vals, rhs, sol, rel_tol, max_iter, stream=None):
    """Allocation-free PCG on caller-provided device arrays (see bal.h): for
    callers that cannot allocate GPU memory while they run. D [nv*9], rows /
    cols int32 [nnz] (rows > cols), vals [nnz*9], rhs / sol [nv*3]."""
    import torch
    nv = D.numel() // 9
    nnz = rows.numel()
    info = SolveInfo()
    _check(load().bal_pcg_solve_noalloc(
        int(nv), _dev(D, torch.float64), int(nnz),
        _dev(rows, torch.int32) if nnz else None, _dev(cols, torch.int32) if nnz else None,
        _dev(vals, torch.float64) if nnz else None, _dev(rhs, torch.float64, 3 * nv),
        _dev(sol, torch.float64, 3 * nv), float(rel_tol), int(max_iter), C.byref(info),
        _stream(stream)))
    return _as_dict(info)


def pair_key(kind, a, b):
    return (int(kind) << 62) | (int(a) << 31) | int(b)


def unpack_key(k):
    k = int(k)
    return (k >> 62, (k >> 31) & 0x7FFFFFFF, k & 0x7FFFFFFF)
