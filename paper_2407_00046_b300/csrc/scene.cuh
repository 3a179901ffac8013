// Internal scene state of libbal and the host-side launchers of each kernel
// family. Everything here is private to the library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace bal {

// Device buffer with a capacity (bytes); grown with cudaMalloc outside the hot loop.
struct Buf {
  void* p = nullptr;
  size_t cap = 0;
  template <typename T>
  T* as() const { return reinterpret_cast<T*>(p); }
};
bal_status buf_reserve(Buf& b, size_t bytes);
void buf_free(Buf& b);

// Pair keys: (kind << 62) | (first << 31) | second.
__host__ __device__ inline uint64_t pair_key(int kind, uint32_t a, uint32_t b) {
  return ((uint64_t)kind << 62) | ((uint64_t)a << 31) | (uint64_t)b;
}
__host__ __device__ inline int key_kind(uint64_t k) { return (int)(k >> 62); }
__host__ __device__ inline uint32_t key_a(uint64_t k) { return (uint32_t)((k >> 31) & 0x7fffffffu); }
__host__ __device__ inline uint32_t key_b(uint64_t k) { return (uint32_t)(k & 0x7fffffffu); }

// Per-pair flags of the evaluation list (A union A').
enum : uint8_t { PF_A = 1, PF_AP = 2 };

// Device-resident PCG scalars (one solve at a time per scene).
struct PcgScalars {
  double rz, pq, alpha, beta;
  double r0norm, rnorm, bnorm, best;
  double tol_abs;
  int32_t it, best_it, done, stagnated, converged, max_it, window, pad;
  uint32_t counter;   // last-block counter of the fused reductions
  uint32_t counter2;
  float alpha_hi, alpha_lo, beta_hi, beta_lo;   // alpha, beta as double-floats
  double stall_rel;   // the stagnation window may end the solve only once ||r|| <= stall_rel ||r_0||
};

// Plain-old-data view of the scene's fixed device arrays, passed by value to kernels.
struct Dev {
  int32_t nv = 0, nt = 0, nf = 0, ne = 0, nsv = 0;
  int64_t nnzL = 0;
  double h = 0, dhat = 0;
  // topology + rest data
  const int32_t *tets = nullptr, *tris = nullptr, *edges = nullptr, *surf = nullptr;
  const uint8_t* pinned = nullptr;
  const double *Dm_inv = nullptr, *vol = nullptr, *mu = nullptr, *lam = nullptr, *mass = nullptr;
  const double* edge_l2 = nullptr;   // [ne] rest squared length of each surface edge (EE mollifier)
  // static lower pattern: CSR + per-block row, element -> slot map
  const int32_t *L_row_ptr = nullptr, *L_col = nullptr, *L_row = nullptr;
  const int32_t* tet_slot = nullptr;  // [nt][6]: 2*slot + (1 if the stored block is the transpose)
  // assembled matrix
  double *D = nullptr, *Dinv = nullptr, *Lval = nullptr, *Lambda = nullptr;
  // step vectors
  double* y = nullptr;
};

struct Scene {
  Dev d;
  int32_t& nv() { return d.nv; }
  double grav[3] = {0, 0, 0};
  double mean_edge = 0;   // mean rest surface edge length (grid cell sizing)
  double mbar = 0;        // mean lumped mass
  bal_params prm{};
  int64_t pair_limit = 0;
  std::vector<double> mass_h;
  std::vector<int32_t> row_ptr_h, col_h;
  std::vector<void*> owned;   // fixed device allocations freed at destroy

  // contact part of the matrix
  int64_t nnzC = 0;
  Buf C_row, C_col, C_val, C_val32;
  // FP32 copies for the mixed-precision solve (valid after make_f32_copy)
  float *D32 = nullptr, *Dinv32 = nullptr, *Lval32 = nullptr;
  float *b32 = nullptr, *x32 = nullptr, *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr;
  bool f32_valid = false;
  int32_t f32_form = -1;         // bal_mixed_operator the FP32 copy was built in
  Buf f32_S;                     // FP64 sums of the difference form's diagonal blocks [nv][9]
  Buf add_inv;                   // additive preconditioner: inverses of the 27x27 group blocks
  // BAL_PREC_DF64 solve (ddpcg.cu). The static lower blocks in a symmetric
  // sliced-ELL layout of 32-row slices, built on first use: per slice the
  // row-side list (blocks L_ij of the slice's rows, k-major: entry k of the 32
  // rows adjacent) and the column-side list (for row i the blocks L_ki with
  // k > i, as value positions into the row-side storage plus the source row);
  // padding entries point at zero blocks.
  int32_t n_slices = 0;
  bool sell_built = false;
  int32_t sell_window = 0;     // spmv_window the layout was built for
  Buf sell_offR, sell_offT;   // [n_slices+1] entry offsets (multiples of 32)
  Buf sell_Rcol;              // [offR[n]] column of each row-side entry
  Buf sell_Tpos, sell_Tsrc;   // [offT[n]] value position / source row of each column-side entry
  Buf sell_pos;               // [nnzL] value position of each CSR slot
  Buf sell_len;               // [n_slices*32] short2: row-side, column-side list length per slot
  Buf sell_srow, sell_slot;   // slot -> row (-1: none) and row -> slot: rows sorted by list length
                              // within windows of 4096 (sliced ELL with a sorting window)
  int64_t sell_zero = 0;      // value position of the chunk of zero blocks (padding)
  // double-float values (valid after the refresh in pcg_df64): slice-major D,
  // D^-1 ([n_slices][9][32]), the sliced lower blocks, contact blocks [nnzC][9],
  // six vectors x r z p q b
  Buf dd_D, dd_Dinv, dd_R, dd_C, dd_vec;
  bool dd_valid = false;
  // contact rows (per assembly): unique rows touched by C or C^T, their entries
  // (2c + transposed) and source vertices in CSR form
  int32_t n_crows = 0;
  Buf cr_rows, cr_ptr, cr_ent, cr_src;
  // their build (rows_bucket): keys vertex << 32 | entry, bucket scratch,
  // ordered entry indices, per-vertex counts / offsets / entries, row positions
  Buf cr_key, cr_bucket, cr_sorted, cr_cnt, cr_off, cr_len, cr_rpos;
  Buf cr_of, cr_q;               // vertex -> contact row (-1: none); contact part of H p per contact row
  bool assembled = false;
  bool project = true;           // PSD projection of stencil Hessians (false: adjoint)
  double* E = nullptr;           // [nt] Young's modulus (device)
  std::vector<double> E_h, nu_h;

  // contact emission + sort scratch
  Buf emit_keys, emit_vals;      // contact blocks as emitted: [n][6] keys, [n][6][9] values
  // duplicate-block merge (segreduce.cu): per-row counts / offsets, buckets,
  // ordered record indices, distinct-column counts / offsets, scan tile sums
  Buf cm_cnt, cm_off, cm_bucket, cm_sorted, cm_ucnt, cm_uoff, scan_aux;
  Buf cub_tmp;

  // broad phase scratch
  Buf bp_cells, bp_cells_alt, bp_ids, bp_ids_alt, bp_count, bp_offs;
  // LBVH (lbvh.cu): primitive boxes, node boxes, keys, children, parents, leaf
  // primitives, refit arrival counters, centre bounds
  Buf lb_pbox, lb_nbox, lb_keys, lb_keys_alt, lb_child, lb_parent, lb_prim, lb_arrivals, lb_bounds;
  Buf cand, cand_alt;            // candidates at r = dhat (sorted keys)
  int64_t n_cand = 0;
  Buf dist, dist_alt;            // per-pair distances scratch
  Buf flags;                     // per-pair selection flags
  Buf eval_keys, eval_flags, eval_mu, eval_s;   // evaluation list A u A'
  int64_t n_eval = 0;
  // friction (Sec. 4.1) lagged at the last contact-term evaluation: pair keys,
  // closest-point weights [n][4], unit normals [n][3], normal forces [n]
  Buf fr_keys, fr_beta, fr_n, fr_lam;
  int64_t n_fr = 0;
  bool fric_suspend = false;     // sigma0 evaluation: barrier gradient only
  Buf ls_cand, ls_cand_alt;      // line-search candidates
  int64_t n_ls_cand = 0;

  // vectors (device, 3*nv doubles each)
  double *xt = nullptr, *grad = nullptr, *gtmp = nullptr, *xtrial = nullptr, *dir = nullptr;
  double *pcg_r = nullptr, *pcg_z = nullptr, *pcg_p = nullptr, *pcg_q = nullptr, *pcg_x = nullptr;
  double* pnorm = nullptr;       // [nv] |p_v|
  int32_t* group = nullptr;       // [nv] stiffness group of the warm start
  // bodies (connected components of the tet mesh)
  int32_t nbody = 0;
  int32_t* body = nullptr;        // [nv]
  double* body_inv_cnt = nullptr; // [nbody]
  double* bmean = nullptr;        // [nbody][3]
  double* bmot = nullptr;         // [nbody] motion inflation of the inter-body pass
  Buf bstats;                     // per-body deviation bound + AABB (ordered bits)
  // reductions
  double* partials = nullptr;    // [kMaxPartials]
  double* scal = nullptr;        // [64] scalar results
  PcgScalars* pcg = nullptr;

  // per-launch timing of the SpMV kernel of each PCG iteration (bal_kernel_timing)
  static constexpr int kTimedPerChunk = 16;
  bool ktime = false;
  cudaEvent_t kev[2 * kTimedPerChunk] = {};
  double kt_ms = 0;
  int64_t kt_n = 0;
  // the same switch times the assembly: the element Hessian kernel alone
  // (events 0, 1) and the whole assembly (events 2, 3: elastic, contact
  // stencils, duplicate-block merge, D^-1) of every assemble call
  cudaEvent_t kaev[4] = {};
  double ka_elastic_ms = 0, ka_total_ms = 0;
  int64_t ka_n = 0;

  // AL state of the current time step (host copy is authoritative)
  bool step_active = false;
  double sigma = 0, sigma0 = 0, dmin_prev = 0, e0 = 0;
  bool sigma0_pending = false;   // A(x_0) empty: sigma0 taken when contact appears
  int32_t l = 0;
  std::vector<uint64_t> ap_keys;
  std::vector<double> ap_mu;
  Buf ap_keys_d, ap_mu_d, ap_s_d;   // device copy of A' (keys, mu, s fixed in the iteration)
};

constexpr int kMaxPartials = 4096;

// event pair k of the current chunk around the timed kernel (no-ops unless enabled)
inline void kt_before(Scene& S, int k, cudaStream_t st) {
  if (S.ktime) cudaEventRecord(S.kev[2 * k], st);
}
inline void kt_after(Scene& S, int k, cudaStream_t st) {
  if (S.ktime) cudaEventRecord(S.kev[2 * k + 1], st);
}
// after the stream has synchronised: add the first n pairs to the totals
bal_status kt_collect(Scene& S, int n);

// ---- elastic.cu ---------------------------------------------------------------
// grad (+)= inertia + elastic gradient (pinned zeroed); init=true overwrites.
bal_status launch_inertia_elastic_grad(Scene& S, const double* x, double* grad,
                                       cudaStream_t st);
// D = m/h^2 I, Lval = 0, Lambda = m/h^2; then element Hessian blocks (projected)
// and their mean eigenvalue into Lambda.
bal_status launch_elastic_assemble(Scene& S, const double* x, cudaStream_t st);
// partial sums of (inertia, elastic) energy and an inversion count; result in
// S.scal[0] (inertia), S.scal[1] (elastic), S.scal[2] (number of tets with J <= 0).
bal_status launch_elastic_energy(Scene& S, const double* x, cudaStream_t st);
// acc[e] += -lam_e^T grad W_e / E_e
bal_status launch_dLdE(Scene& S, const double* x, const double* lam_adj, double* acc, cudaStream_t st);

// ---- contact.cu ---------------------------------------------------------------
// distances of n pairs (keys) at x into d (device).
bal_status launch_pair_distance(Scene& S, const double* x, const uint64_t* keys, int64_t n,
                                double* d, cudaStream_t st);
// gradient (+=) and, if hess, projected Hessian blocks of the eval list.
bal_status launch_contact_terms(Scene& S, const double* x, double* grad, bool hess,
                                cudaStream_t st);
// sum over eval-like arrays of phi (barrier for A members at d<dhat, AL for A').
// Writes S.scal[slot] = contact energy, S.scal[slot+1] = count of d < dhat over keys.
bal_status launch_contact_energy(Scene& S, const double* x, const uint64_t* cand, int64_t ncand,
                                 int slot, cudaStream_t st);
// min over candidates of step_bound*d/Delta_i (where step_bound*d < Delta_i), with
// Delta_i = max |p_a - p_b| over a node of each primitive -> S.scal[slot].
bal_status launch_step_bound(Scene& S, const double* x, const double* dir,
                             const uint64_t* cand, int64_t ncand, int slot, cudaStream_t st);
// min over candidates of the conservative time of impact of the cubic CCD
// (Sec. 5.3) along x + t dir, t in [0, 1] -> S.scal[slot].
bal_status launch_ccd_bound(Scene& S, const double* x, const double* dir,
                            const uint64_t* cand, int64_t ncand, int slot, cudaStream_t st);
// flag[i] = candidate i can enter A along the step or constrain alpha
bal_status launch_ls_filter(Scene& S, const double* x, const double* dir, const uint64_t* cand,
                            int64_t n, uint8_t* flag, cudaStream_t st);
bal_status launch_flag_below(const double* d, int64_t n, double thr, uint8_t* flag, cudaStream_t st);
// A' dual update: s_i, mu_i += sigma b(d_i, dhat + s_i) for the device A' list.
bal_status launch_dual_update(Scene& S, const double* x, int64_t n, cudaStream_t st);

// ---- broadphase.cu -------------------------------------------------------------
// All PT/EE pairs whose primitives' (AABB) distance can be below r, sorted, in
// out (grown as needed). Returns the count in *n.
bal_status find_candidates(Scene& S, const double* x, double r, Buf& out, Buf& alt,
                           int64_t* n, cudaStream_t st);
// Every pair that can satisfy step_bound*d < Delta or d < dhat + Delta along
// x + alpha dir (alpha <= 1), Delta = max |p_a - p_b|: displacements are split
// into a per-body mean and a deviation; same-body pairs are inflated by the
// deviations only, different-body pairs also by |mean|.
bal_status find_candidates_motion(Scene& S, const double* x, const double* dir, Buf& out,
                                  Buf& alt, int64_t* n, cudaStream_t st);

// ---- lbvh.cu ---------------------------------------------------------------------
// PT / EE pairs whose (swept, if dir) primitive boxes come within r on every
// axis, from linear BVHs over the surface triangles and edges; sorted keys.
bal_status lbvh_candidates(Scene& S, const double* x, const double* dir, double r, Buf& out, Buf& alt,
                           int64_t* n, cudaStream_t st);

// ---- matrix.cu -----------------------------------------------------------------
bal_status contact_blocks_reduce(Scene& S, int64_t n_emit, cudaStream_t st);
bal_status scan_i32(Scene& S, const int32_t* in, int32_t* out, int64_t n, cudaStream_t st);
bal_status rows_bucket(Scene& S, const uint64_t* keys, int64_t n, int nv, int32_t* cnt, int32_t* off,
                       int32_t* bucket, int32_t* sorted, int32_t* ucnt, cudaStream_t st);
bal_status launch_dinv(Scene& S, cudaStream_t st);
bal_status spmv(Scene& S, const double* v, double* y, cudaStream_t st);
bal_status spmv32(Scene& S, const float* v, float* y, cudaStream_t st);
bal_status make_f32_copy(Scene& S, cudaStream_t st);
// order-preserving stream compaction of flagged entries (count read back)
bal_status compact_u64(Scene& S, const uint64_t* in, const uint8_t* flag, int64_t n, uint64_t* out,
                       int64_t* nsel, cudaStream_t st);
bal_status compact_f64(Scene& S, const double* in, const uint8_t* flag, int64_t n, double* out,
                       int64_t* nsel, cudaStream_t st);
// S.scal[8] = ||b - y||^2, S.scal[9] = ||b||^2
bal_status launch_residual_norm(Scene& S, const double* b, const double* y, cudaStream_t st);
bal_status pcg_solve(Scene& S, const double* b, double* x, double tol, int max_it,
                     bal_solve_info* info, cudaStream_t st);
// x = H^{-1} b by block-Jacobi PCG with double-float recurrences (ddpcg.cu):
// FP64 true residuals decide convergence; restarts from the true residual when
// the recurrence and the true residual disagree.
bal_status pcg_df64(Scene& S, const double* b, double* x, double tol, int max_it,
                    bal_solve_info* info, cudaStream_t st);
// S.scal[8] = ||b - H x||^2, S.scal[9] = ||b||^2 and r = b - H x (FP64)
bal_status residual_fp64(Scene& S, const double* b, const double* x, double* r, double* rn,
                         double* bn, cudaStream_t st);

// ---- vec.cu ----------------------------------------------------------------------
bal_status launch_make_y(Scene& S, const double* xt, const double* vt, double* y, cudaStream_t st);
// out = y + a x over n doubles
bal_status launch_axpy(Scene& S, int64_t n, double a, const double* x, const double* y, double* out,
                       cudaStream_t st);
bal_status launch_dot(Scene& S, int64_t n, const double* a, const double* b, int slot, cudaStream_t st);
// S.scal[slot] = max, S.scal[slot + 1] = min of Lambda over free DOFs
bal_status launch_lambda_range(Scene& S, int slot, cudaStream_t st);
// S.scal[slot] = max over surface vertices of |d_v|
bal_status launch_surf_max_norm(Scene& S, const double* d, int slot, cudaStream_t st);

// ---- reductions helper (matrix.cu) -----------------------------------------------
// S.scal[slot] = sum / min / max of partials[0..n)
enum RedOp { RED_SUM = 0, RED_MIN = 1, RED_MAX = 2 };
bal_status finish_reduce_offset(Scene& S, int offset, int n, int slot, RedOp op, cudaStream_t st);
inline bal_status finish_reduce(Scene& S, int n, int slot, RedOp op, cudaStream_t st) {
  return finish_reduce_offset(S, 0, n, slot, op, st);
}

}  // namespace bal
