/*
 * libbal -- C ABI of the barrier-augmented Lagrangian (BAL) inexact Newton-PCG
 * time step of "Barrier-Augmented Lagrangian for GPU-based Elastodynamic
 * Contact" (arXiv 2407.00046), hand-written CUDA for sm_103a (B300).
 *
 * Conventions shared by every entry point
 *   - Positions, velocities and gradients are FP64 arrays [n_verts][3]
 *     (x0 y0 z0 x1 y1 z1 ...), row-major, in DEVICE memory owned by the caller,
 *     unless a parameter says "host".
 *   - Every call that launches work takes a cudaStream_t (passed as void*, NULL
 *     = legacy default stream); all work of the call is ordered on that stream.
 *     Calls that return host-visible results (counts, norms, decisions)
 *     synchronise that stream before returning.
 *   - Errors are returned as bal_status, never thrown, printed or trapped. A
 *     non-OK status leaves the scene usable; bal_last_error() returns a message
 *     describing the calling thread's last failure.
 *   - A bal_scene is not thread-safe: one call at a time per scene.
 */
#ifndef BAL_H_
#define BAL_H_

#include <stdint.h>

#if defined(__GNUC__)
#define BAL_API __attribute__((visibility("default")))
#else
#define BAL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BAL_OK = 0,
  BAL_ERR_ARG = 1,            /* invalid argument / size / pointer */
  BAL_ERR_CAPACITY = 2,       /* a contact buffer exceeded its hard limit */
  BAL_ERR_NOT_CONVERGED = 3,  /* Newton loop hit newton_max_iter */
  BAL_ERR_NAN = 4,            /* NaN / Inf in a gradient, residual or energy */
  BAL_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up */
  BAL_ERR_CUDA = 6,           /* a CUDA runtime call failed */
  BAL_ERR_LINE_SEARCH = 7,    /* step length fell below ls_min_alpha */
  BAL_ERR_STATE = 8           /* call order violated (e.g. solve before assemble) */
} bal_status;

/* FP64: every PCG operation in FP64. MIXED: FP32 inner PCG with FP64 iterative
 * refinement -- each pass solves H e = r / ||r|| in FP32 (mixed_inner_tol,
 * mixed_inner_max) and is kept if it lowers the FP64 quadratic model
 * x^T H x / 2 - b^T x (its change -d.(r + r_new)/2 formed from the correction d
 * and the two FP64 residuals) or the FP64 residual; a pass that lowers neither
 * is rolled back and ends the solve. DF64: PCG recurrences in double-float arithmetic (pairs of FP32,
 * ~47-bit significand) with FP64 residuals deciding convergence; falls back to
 * FP64 for a matrix with an entry beyond 1e36. */
/* FP32: the single-precision path (the paper's single-precision version,
 * Sec. 6): element stencil eigensystems evaluated in FP32 arithmetic, plus the
 * MIXED solver (FP32 matrix copy, SpMV, preconditioner and PCG vectors, FP64
 * refinement). Contact distances, barrier derivatives, the gradient, the
 * residual norms and the line-search energies stay FP64. */
typedef enum { BAL_PREC_FP64 = 0, BAL_PREC_MIXED = 1, BAL_PREC_DF64 = 2, BAL_PREC_FP32 = 3 } bal_precision;
/* The FP32 operator of the FP32 + FP64-refinement solves (BAL_PREC_MIXED,
 * BAL_PREC_FP32; no counterpart in the paper, whose solver is FP64).
 * DIFFERENCE: (H v)_i = G_i v_i + sum_j B_ij (v_j - v_i), with
 * G_i = D_i + the sum of row i's off-diagonal blocks summed in FP64 before its
 * one rounding (m_i/h^2 I wherever every block of the row is translation
 * invariant) -- the form stays exactly translation invariant in FP32, so
 * rounding the blocks of a stiff body leaves its translations exact (its
 * rotations keep an error from rounding the FP32 vector itself).
 * PLAIN: D_i v_i + sum_j B_ij v_j with every block rounded to FP32. */
typedef enum { BAL_MIXED_OP_DIFFERENCE = 0, BAL_MIXED_OP_PLAIN = 1 } bal_mixed_operator;
/* BJ: block-Jacobi. BJ_WARMSTART: block-Jacobi after the stiffness-grouped
 * warm start (Sec. 4.2.2). ADDITIVE: the two-level additive preconditioner the
 * paper compares against (App. A): 3x3 diagonal-block inverses plus exact
 * inverses of the 27x27 blocks of 9 consecutive vertices; always FP64. */
typedef enum { BAL_PRECOND_BJ = 0, BAL_PRECOND_BJ_WARMSTART = 1, BAL_PRECOND_ADDITIVE = 2 } bal_precond;

/* Solver and schedule parameters. bal_default_params follows the paper: Newton
 * tolerance 1e-4 relative (Alg. 1 / Sec. 1 footnote), PCG 1e-4 relative with a
 * 100-iteration stagnation window (App. B), A' threshold 1e-2 dhat, sigma <-
 * max(1.2 sigma, 100 sigma0) while min d < 1e-2 dhat (Alg. 1, Sec. 3.4),
 * alpha_min 1e-9 with rounds of 100 more PCG iterations below it (App. B). */
typedef struct {
  int32_t precision;          /* bal_precision */
  int32_t precond;            /* bal_precond */
  double pcg_tol;             /* ||r_k|| <= pcg_tol ||r_0|| */
  int32_t pcg_max_iter;
  int32_t pcg_stall_window;   /* stop if no new minimum residual in this many iterations */
  double newton_tol;          /* ||e^l||_2 <= newton_tol ||e^0||_2 */
  double newton_abs_tol;      /* or ||e^l||_2 <= newton_abs_tol */
  int32_t newton_max_iter;
  double ap_ratio;            /* A' threshold factor (1e-2) */
  double sigma_growth;        /* 1.2 */
  double sigma_cap;           /* 100: multiple of sigma0 in the sigma schedule */
  int32_t sigma_literal_max;  /* 1 (default) = the printed max(1.2 s, 100 s0) rule of Alg. 1;
                                 0 = the capped reading min(1.2 s, 100 s0) */
  double step_bound;          /* 0.9: CA keeps (1 - step_bound) of each gap; CCD: margin on the TOI */
  double ls_min_alpha;        /* 1e-9 (App. B) */
  double ls_slack;            /* relative energy slack for rounding noise (1e-12) */
  int64_t contact_cap;        /* Sec. 5.2 memory limit on |A| (line-search halving) */
  int32_t ls_extra_pcg;       /* App. B: extra PCG iterations when alpha < ls_min_alpha */
  double warm_tol;            /* warm-start subdomain PCG relative tolerance (1e-2) */
  int32_t warm_max_iter;      /* warm-start subdomain PCG iteration cap (50) */
  int32_t mixed_inner_max;    /* FP32 inner PCG iterations per refinement pass (3000) */
  double mixed_inner_tol;     /* FP32 inner relative tolerance per pass (1e-2) */
  int32_t mixed_max_refine;   /* max FP64 refinement passes, and max restarts from the FP64
                                 residual of the FP64 / DF64 solves (40) */
  int32_t ca_max_iter;        /* step bound: conservative-advancement iterations per pair (64) */
  int32_t freeze_al;          /* 1: hold sigma, A', mu fixed (no dual update, no sigma schedule,
                                 no A' rule) -- the map the adjoint differentiates */
  int32_t step_mode;          /* bal_step_mode: line-search step bound */
  int32_t broad_phase;        /* bal_broad_phase: candidate search */
  int32_t al_mode;            /* bal_al_mode: Algorithm 1, or the plain inexact Newton ablation */
  int32_t pcg_tol_mode;       /* bal_pcg_tol_mode: per-solve PCG tolerance rule */
  double friction;            /* chi of Sec. 4.1 (>= 0; 0 = frictionless). Fully-implicit
                                 friction: every pair of A u A' adds chi lambda f(|w|) with
                                 the normal force lambda, the contact normal and the
                                 closest-point weights lagged at each Newton iterate */
  double friction_eps_v;      /* mollifier threshold eps_v (m/s; 0 = dhat, Table 1 caption);
                                 the static zone is |tangent slip| < eps_v h */
  int32_t spmv_window;        /* double-float SpMV layout: 0 = one thread per row gathering
                                 every transposed block through its column-side list; W > 0
                                 (a multiple of 32, at most 4096) = one CTA per window of W
                                 consecutive rows, transposed blocks of rows in the same
                                 window summed in shared memory (FP64), only the other
                                 windows' through the column-side list */
  int32_t ls_extra_rounds;    /* App. B: rounds of ls_extra_pcg more PCG iterations tried while
                                 the line search ends below ls_min_alpha (then failure) */
  double pcg_stall_forcing;   /* eta > 0: the stagnation window may end a solve only once
                                 ||r|| <= eta ||r_0|| (otherwise the cap or the tolerance ends
                                 it), so an inexact Newton direction reduces the linearised
                                 residual at least by eta; 0 (default) = the window alone */
  int32_t mixed_operator;     /* bal_mixed_operator: form of the FP32 copy of H (DIFFERENCE) */
} bal_params;

/* AL: Algorithm 1 (dual updates, sigma schedule, A' rule). PLAIN: the plain
 * inexact Newton method the paper ablates against -- the barrier with sigma
 * held at sigma0, A' empty, no dual update. */
typedef enum { BAL_AL_ALGORITHM1 = 0, BAL_AL_PLAIN = 1 } bal_al_mode;
/* FIXED: ||r|| <= pcg_tol ||r_0|| on every solve. TRUNCATED_NEWTON: App. B
 * criterion (i), ||r|| <= min(0.5, sqrt(||e||)) ||e|| with e the gradient.
 * COND_X / COND_B: App. B criteria (ii) ||r|| <= u kappa ||x_k|| and (iii)
 * ||r|| <= u kappa ||b|| with u = DBL_EPSILON, x_k the Newton iterate, b = -e
 * and kappa = max / min of the assembled eigenvalue stiffness Lambda over free
 * DOFs (elastic, contact and friction stencils plus the lumped mass); the
 * relative tolerance these give is capped at 0.5. */
typedef enum {
  BAL_PCG_TOL_FIXED = 0,
  BAL_PCG_TOL_TRUNCATED_NEWTON = 1,
  BAL_PCG_TOL_COND_X = 2,
  BAL_PCG_TOL_COND_B = 3
} bal_pcg_tol_mode;

/* Step bound of the line search. CA: conservative advancement on the distance
 * (every pair keeps (1 - step_bound) of its gap). CCD: the cubic CCD of
 * Sec. 5.3 -- coplanarity roots by Newton-bisection with deflation, activation
 * d_TOC < dhat + 1e-12 (a touch, d_TOC < 1e-12, for a pair already within
 * dhat), time of impact backtracked by 0.9 until the triple product keeps the
 * sign of the reference frame, then scaled by step_bound. */
typedef enum { BAL_STEP_CA = 0, BAL_STEP_CCD = 1 } bal_step_mode;
/* Candidate search. GRID: uniform grid hash. LBVH: linear BVHs over triangles
 * and edges (Sec. 5.3, broad phase). */
typedef enum { BAL_BROAD_GRID = 0, BAL_BROAD_LBVH = 1 } bal_broad_phase;

/* Scene description: HOST arrays, copied by bal_create_scene. */
typedef struct {
  int32_t n_verts, n_tets, n_tris, n_edges, n_surf_verts;
  const double* X;            /* [n_verts][3] rest positions (m) */
  const int32_t* tets;        /* [n_tets][4] positively oriented */
  const int32_t* tris;        /* [n_tris][3] boundary triangles */
  const int32_t* edges;       /* [n_edges][2] boundary edges, i < j, sorted unique */
  const int32_t* surf_verts;  /* [n_surf_verts] boundary vertices */
  const double* E;            /* [n_tets] Young's modulus (Pa) */
  const double* nu;           /* [n_tets] Poisson ratio */
  const double* rho;          /* [n_tets] density (kg/m^3) */
  const uint8_t* pinned;      /* [n_verts] 1 = Dirichlet vertex */
  double h;                   /* time step (s) */
  double dhat;                /* contact offset (m) */
  double gravity[3];          /* m/s^2 */
  int64_t pair_capacity;      /* initial candidate-pair buffer (grows up to pair_limit) */
  int64_t pair_limit;         /* hard limit; exceeding it returns BAL_ERR_CAPACITY */
} bal_scene_desc;

typedef struct bal_scene bal_scene;

/* Read-only view of the assembled Hessian in symmetric lower storage
 * H = D + L + L^T + C + C^T (Sec. 5.1, App. C): D = 3x3 diagonal blocks
 * [n_verts][9]; L = static lower blocks in CSR (row_ptr[n_verts+1], col[nnz_L],
 * val[nnz_L][9]); C = merged contact lower blocks (row[nnz_C], col[nnz_C],
 * val[nnz_C][9]) sorted by (row, col). Blocks are row-major 3x3; a lower block
 * at (row i, col j), i > j, holds H[3i..3i+2, 3j..3j+2]. Device pointers owned
 * by the scene, valid until the next assemble call. */
typedef struct {
  int32_t n_verts;
  int64_t nnz_L, nnz_C;
  const double* D;
  const int32_t* L_row_ptr;
  const int32_t* L_col;
  const double* L_val;
  const int32_t* C_row;
  const int32_t* C_col;
  const double* C_val;
  const double* Lambda;       /* [n_verts][3] assembled eigenvalue stiffness (Sec. 4.2.2) */
} bal_bsr_view;

/* Augmented-Lagrangian state of the current time step (Alg. 1). Arrays are
 * HOST arrays. A pair key packs (kind << 62) | (first << 31) | second with
 * kind 0 = point-triangle (vertex id, triangle index) and kind 1 = edge-edge
 * (edge index, edge index, first < second). */
typedef struct {
  double sigma, sigma0;
  double dmin_prev;
  int64_t n_ap;               /* |A'| */
  uint64_t* ap_keys;          /* [n_ap] sorted ascending */
  double* ap_mu;              /* [n_ap] */
} bal_al_state;

typedef struct {
  int32_t iters;              /* PCG iterations performed */
  double rel_residual;        /* ||b - H x|| / ||b||, recomputed in FP64 */
  double rel_residual_r0;     /* ||b - H x|| / ||r_0|| */
  int32_t stagnated;          /* 1 if stopped by the stagnation window */
  int32_t converged;          /* 1 if the tolerance was met */
  int32_t refine_passes;      /* mixed: FP64 refinement passes; FP64 / df64: restarts from the FP64 residual */
  int32_t warm_iters;         /* warm start: subdomain PCG iterations */
  int32_t n_groups;           /* warm start: stiffness groups */
  int32_t negative_curvature; /* adjoint: 1 if the unprojected H was indefinite and the
                                 projected H was used instead */
  int32_t precision_used;     /* bal_precision the solve ran in */
} bal_solve_info;

typedef struct {
  int32_t l;                  /* iteration index inside the time step */
  int32_t converged;          /* 1 if the convergence test passed (no step taken) */
  int64_t n_active;           /* |A| at the iterate */
  int64_t n_ap;               /* |A'| */
  int64_t n_candidates;       /* line-search candidate pairs */
  double dmin;                /* min distance over A (inf if empty) */
  double sigma;
  double grad_norm;           /* ||e^l||_2 */
  double alpha;               /* accepted step length (0 if none) */
  int32_t ls_trials;
  int32_t pcg_iters;
  double pcg_rel_residual;
  double energy;              /* L_sigma at the accepted iterate */
  double ms_assemble, ms_solve, ms_line_search, ms_contact;
  double ms_ls_broad, ms_ls_bound, ms_ls_energy;   /* line-search breakdown */
  int64_t n_raw_candidates;   /* line-search pairs from the broad phase, before filtering */
  double pcg_tol;             /* relative PCG tolerance the solve used */
  double kappa;               /* Lambda max / min over free DOFs (COND_X / COND_B; else 0) */
} bal_newton_info;

typedef struct {
  int32_t newton_iters;
  int32_t pcg_iters_total;
  int32_t converged;
  int64_t max_active;
  double min_distance;        /* min d over A seen at the iterates */
  double sigma0, sigma_final;
  double ms_total, ms_assemble, ms_solve, ms_line_search, ms_contact;
} bal_step_info;

/* ---- lifetime ------------------------------------------------------------ */
BAL_API const char* bal_last_error(void);
/* Number of CUDA kernels this library has launched in the process so far
 * (its own kernels; library sort / scan kernels are not counted). */
BAL_API uint64_t bal_launch_count(void);
/* sizeof of this build's ABI structs, for bindings to check their mirrors
 * (no paper counterpart): which = 0 bal_params, 1 bal_scene_desc,
 * 2 bal_bsr_view, 3 bal_al_state, 4 bal_solve_info, 5 bal_newton_info,
 * 6 bal_step_info; 0 for any other value. Host-only, needs no GPU. */
BAL_API uint64_t bal_struct_size(int32_t which);
BAL_API void bal_default_params(bal_params* out);

/* Copies the topology, precomputes D_m^{-1}, rest volumes, Lame parameters and
 * lumped masses (Sec. 3.1), and builds the static lower BSR pattern with its
 * element-to-slot map (Sec. 5.1, App. C). Allocates the scene's device
 * buffers on the current device. */
BAL_API bal_status bal_create_scene(const bal_scene_desc* desc, const bal_params* params,
                            bal_scene** out);
BAL_API bal_status bal_destroy_scene(bal_scene* scene);
BAL_API bal_status bal_set_params(bal_scene* scene, const bal_params* params);
/* Per-launch timing of the SpMV kernel of every PCG iteration (the dominant
 * kernel of a solve: the off-diagonal product of the FP64 / mixed solvers, the
 * gather product of the double-float one) with CUDA events recorded on the
 * solve's stream. Returns in total_ms / launches (either may be NULL) the sum
 * of the durations and the number of timed launches since the previous call,
 * resets both, and enables (enable != 0) or disables timing for later solves.
 * Not in the paper: measurement support. */
BAL_API bal_status bal_kernel_timing(bal_scene* scene, int32_t enable, double* total_ms,
                                     int64_t* launches);
/* FP64 FMA throughput of the current device in TFLOP/s (2 flop per FMA), from
 * one timed launch of `iters` FMA rounds on 8 independent chains per thread
 * over 8 CTAs of 256 threads per SM: the ALU ceiling of the FP64 kernels.
 * Allocates and frees a small scratch buffer on `stream`. Not in the paper:
 * measurement support. */
BAL_API bal_status bal_fp64_fma_rate(int32_t iters, double* tflops, void* stream);
/* Assembly timing under the same switch: per assemble call, CUDA events on
 * its stream around the element Hessian kernel and around the whole assembly
 * (element stencils, contact stencils, duplicate-block merge, D^-1). Returns
 * the sums since the previous call (either pointer may be NULL) and the
 * number of timed assemblies, and resets them. Not in the paper:
 * measurement support. */
BAL_API bal_status bal_assembly_timing(bal_scene* scene, double* elastic_ms, double* total_ms,
                                       int64_t* assemblies);

BAL_API bal_status bal_get_params(const bal_scene* scene, bal_params* out);
/* Host copies of the static pattern: row_ptr [n_verts+1], col [nnz_L]; either
 * may be NULL to query nnz only. */
BAL_API bal_status bal_static_pattern(const bal_scene* scene, int64_t* nnz_L, int32_t* row_ptr,
                              int32_t* col);
/* Lumped masses [n_verts] (host out). */
BAL_API bal_status bal_get_mass(const bal_scene* scene, double* mass_host);

/* ---- time step state ------------------------------------------------------ */
/* Starts a time step from (x_t, v_t) (device): y = x_t + h v_t + h^2 g
 * (Sec. 3.1), A at x_t, sigma0 (Sec. 3.4), mu = 0, A' empty. */
BAL_API bal_status bal_step_begin(bal_scene* scene, const double* x_t, const double* v_t,
                          void* stream);
/* AL state of the current step. ap_keys / ap_mu may be NULL to query n_ap;
 * otherwise they must hold `capacity` entries. */
BAL_API bal_status bal_get_al_state(const bal_scene* scene, bal_al_state* out, int64_t capacity);
/* Replaces sigma, sigma0, dmin_prev and A' (host keys sorted ascending). */
BAL_API bal_status bal_set_al_state(bal_scene* scene, const bal_al_state* in);
/* Inertia target y of the current step into y_out (device). */
BAL_API bal_status bal_get_y(const bal_scene* scene, double* y_out, void* stream);

/* ---- hot-path calls --------------------------------------------------------- */
/* Assembles at x (device) the gradient e = grad L_sigma (Eq. aug-lag; pinned
 * entries zero) into grad_out (device, may be NULL) and the PSD-projected
 * Hessian (elements: projection of dP/dF; contact stencils: projection of the
 * 12x12 stencil Hessian; Sec. 4.2.2) into scene storage, with A = {d < dhat}
 * found at x and A', mu, sigma from the current step state; s_i evaluated at x
 * (Sec. 3.2.2). Pinned rows and columns are eliminated with diagonal m/h^2
 * (App. C). Fills *view if non-NULL. */
BAL_API bal_status bal_assemble_hessian(bal_scene* scene, const double* x, double* grad_out,
                                bal_bsr_view* view, void* stream);
/* Copies the last assembled Hessian into caller-owned DEVICE buffers (any may
 * be NULL): D [n_verts*9], L values [nnz_L*9], contact rows/cols [nnz_C],
 * contact values [nnz_C*9], Lambda [n_verts*3]. Sizes are those reported in
 * bal_bsr_view by the assemble call. */
BAL_API bal_status bal_copy_hessian(bal_scene* scene, double* D_out, double* L_val_out,
                                    int32_t* C_row_out, int32_t* C_col_out, double* C_val_out,
                                    double* Lambda_out, void* stream);
/* y = H v with the last assembled H (Sec. 5.1 SpMV; device in/out). */
BAL_API bal_status bal_spmv(bal_scene* scene, const double* v, double* y, void* stream);
/* Solves H sol = rhs with block-Jacobi PCG (Sec. 4.2, App. B), optionally
 * warm-started by the stiffness-grouped subdomain solve (Sec. 4.2.2), or in
 * FP32 with FP64 iterative refinement, from sol_inout. Stops at
 * ||r_k|| <= rel_tol ||r_0||, when the residual reaches no new minimum in
 * pcg_stall_window iterations, or at max_iter. In the FP64 (block-Jacobi or
 * additive) and DF64 forms the FP64 residual b - H x decides convergence:
 * when the recursion reports it but
 * the FP64 residual is still above rel_tol ||r_0||, CG restarts from the FP64
 * residual (at most mixed_max_refine times; info->refine_passes counts them). */
BAL_API bal_status bal_pcg_solve(bal_scene* scene, const double* rhs, double* sol_inout,
                         double rel_tol, int32_t max_iter, bal_solve_info* info,
                         void* stream);
/* L_sigma at x with A(x) and the step's A' state (host out). */
BAL_API bal_status bal_energy(bal_scene* scene, const double* x, double* energy_out, void* stream);
/* Broad phase (Sec. 5.3): the PT / EE candidate pairs (sorted keys, kind << 62
 * | first << 31 | second) of the scene's broad_phase at x. With dir == NULL:
 * pairs whose primitives' boxes come within r on every axis (a superset of the
 * pairs with d < r). With dir (device [n_verts*3]): the LBVH returns the pairs
 * whose boxes swept from x to x + dir come within r; the grid returns its
 * line-search candidate set (r unused). keys_out: device, capacity entries;
 * *n_out (host) is the count; BAL_ERR_CAPACITY if it exceeds capacity. */
BAL_API bal_status bal_find_candidates(bal_scene* scene, const double* x, const double* dir, double r,
                                       uint64_t* keys_out, int64_t capacity, int64_t* n_out,
                                       void* stream);
/* Line-search step bound along x + t dir, t in [0, 1] (Sec. 5.3 / Sec. 5.2):
 * the minimum over the given pairs (device array of pair keys, kind << 62 |
 * first << 31 | second; kind 0 = PT (vertex, triangle), 1 = EE (edge, edge))
 * of the conservative-advancement bound (mode BAL_STEP_CA) or of the cubic
 * CCD's conservative time of impact (BAL_STEP_CCD), capped at 1. x and dir
 * are device [n_verts*3] FP64; *alpha_out is host. */
BAL_API bal_status bal_step_bound(bal_scene* scene, const double* x, const double* dir,
                                  const uint64_t* pair_keys, int64_t n_pairs, int32_t mode,
                                  double* alpha_out, void* stream);
/* One Alg. 1 iteration l on x_inout (device): dual update of the previous
 * iteration, A, A' rule, gradient and convergence test, assembly, PCG, step
 * bound, backtracking line search (Sec. 5.2 memory cap). */
BAL_API bal_status bal_newton_step(bal_scene* scene, double* x_inout, bal_newton_info* info,
                           void* stream);
/* Ends the current time step at x (device): v_out = (x - x_t) / h (Sec. 3.1),
 * x_t being the state passed to bal_step_begin. v_out is device [n_verts*3]. */
BAL_API bal_status bal_step_end(bal_scene* scene, const double* x, double* v_out, void* stream);
/* Full time step: bal_step_begin + Alg. 1 loop + v = (x - x_t)/h (Sec. 3.1). */
BAL_API bal_status bal_time_step(bal_scene* scene, double* x_inout, double* v_inout,
                         bal_step_info* info, void* stream);

/* ---- allocation-free solve (no counterpart in the paper) -------------------- */
/* For callers that cannot allocate GPU memory while they run (a host
 * application that owns all device memory, or a loop that forbids allocation
 * after start-up): block-Jacobi PCG with the stopping rules of bal_pcg_solve
 * under the default parameters (||r|| <= rel_tol ||r_0||, no new minimum of
 * the preconditioned residual sqrt(r^T z) in 100 iterations, or max_iter)
 * but without its restarts from the FP64 residual (info->rel_residual reports
 * that residual; a caller needing it below rel_tol calls again from sol), on
 * a caller-provided symmetric block matrix
 * H = D + L + L^T in DEVICE memory -- D [n_verts][9] diagonal blocks, nnz lower
 * blocks (rows[nnz], cols[nnz] with rows > cols, vals[nnz][9] row-major) --
 * solving H sol = rhs from the initial guess in sol (device, in/out). It calls
 * no cudaMalloc / cudaFree: its working vectors live in a fixed device array
 * of about 2.8 MB that every GPU loading the library keeps until exit, so
 * n_verts may not exceed BAL_NOALLOC_MAX_VERTS (larger sizes return
 * BAL_ERR_ARG). The first call on a device looks up that array's address and
 * should come before any stream capture; the address is cached per device
 * index for the life of the process, which assumes the device's primary
 * context throughout (no cudaDeviceReset between calls). All calls share the
 * array: calls that overlap on the GPU race and must be serialised by the
 * caller. A non-finite residual or p^T H p <= 0 returns BAL_ERR_NAN. */
#define BAL_NOALLOC_MAX_VERTS 16384
BAL_API bal_status bal_pcg_solve_noalloc(int32_t n_verts, const double* D, int64_t nnz,
                                         const int32_t* rows, const int32_t* cols,
                                         const double* vals, const double* rhs, double* sol,
                                         double rel_tol, int32_t max_iter,
                                         bal_solve_info* info, void* stream);

/* ---- adjoint of the time step (not in the paper) ----------------------------- */
/* Replaces per-tet Young's modulus and Poisson ratio (HOST arrays [n_tets]). */
BAL_API bal_status bal_set_materials(bal_scene* scene, const double* E, const double* nu);

/* Adjoint of one time step x_{t+1} = argmin L_sigma(x; x_t, v_t, E) with the
 * converged AL state `al` (sigma, A', mu of the step's last iteration) held
 * fixed: differentiating grad_x L(x_{t+1}) = 0 gives H lambda = a with H the
 * UNPROJECTED Hessian at x_{t+1} and a = dL/dx_{t+1} + dL/dv_{t+1} / h
 * (v_{t+1} = (x_{t+1} - x_t)/h). Then, on free vertices,
 *   dL/dx_t = M lambda / h^2 - dL/dv_{t+1} / h,   dL/dv_t = M lambda / h,
 * (pinned entries are zero) and dL/dE_e += -lambda_e^T grad W_e / E_e (mu and
 * lam are linear in E). If PCG finds H indefinite it falls back to the
 * projected H and sets info->negative_curvature. All vectors are DEVICE
 * [n_verts*3]; dLdE_accum is DEVICE [n_tets] (accumulated). Overwrites the
 * scene's current step state (y, A', mu, sigma). Frictionless steps only:
 * returns BAL_ERR_ARG when params.friction > 0. */
BAL_API bal_status bal_adjoint_step(bal_scene* scene, const double* x_t, const double* v_t,
                                    const double* x_next, const bal_al_state* al,
                                    const double* dLdx_next, const double* dLdv_next,
                                    double* dLdx_prev, double* dLdv_prev, double* dLdE_accum,
                                    double rel_tol, int32_t max_iter, bal_solve_info* info,
                                    void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BAL_H_ */
