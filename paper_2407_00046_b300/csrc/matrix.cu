// Sparse Hessian storage and the PCG solve (Sec. 5.1, Sec. 4.2, App. B), FP64.
//
// H = D + L + L^T + C + C^T: D dense 3x3 diagonal blocks (also the block-Jacobi
// preconditioner), L the static lower blocks from node adjacency in CSR with a
// per-block row index, C the contact lower blocks rebuilt every assembly. The
// contact blocks are emitted per stencil as (row << 32 | col, 3x3) records,
// radix-sorted by key (stable, so equal keys keep emission order) and summed per
// run of equal keys in a fixed order -- the duplicate-block reduction.
//
// SpMV y = H v: a diagonal pass writes y = D v, then one thread per stored lower
// block adds L_ij v_j to y_i and L_ij^T v_i to y_j with atomic adds (the
// paper's map-reduce with atomic addition over symmetric storage).
//
// PCG runs with every scalar on the device: per iteration three kernels --
// (1) p = z + beta p, q = D p and partial sums of p^T D p; (2) off-diagonal
// blocks into q and partial sums of 2 p_i^T L_ij p_j, the last CTA turning
// p.q = p^T H p into alpha; (3) x += alpha p, r -= alpha q, z = D^{-1} r and
// partial sums of r.z, r.r, the last CTA deciding convergence (||r|| <= tol
// ||r_0||), stagnation (no new minimum of the preconditioned residual
// sqrt(r.z) in `window` iterations: ||r||_2 of CG on a stiff system can rise
// for hundreds of iterations while the iterate improves) and beta. Once `done` is set the remaining launches of a chunk return at once, so
// the host only synchronises once per chunk of iterations.
#include <cub/cub.cuh>
#include <utility>

#include "scene.cuh"

namespace bal {

namespace {

constexpr int kRedBlocks = 8 * kNumSM;   // CTAs of every fused PCG reduction kernel (latency hiding)
constexpr int kRedThreads = 256;

template <int NT>
__global__ void k_finish(const double* __restrict__ partials, int n, double* out, int op) {
  double acc = op == RED_SUM ? 0.0 : (op == RED_MIN ? INFINITY : -INFINITY);
  for (int i = threadIdx.x; i < n; i += NT) {
    const double v = partials[i];
    acc = op == RED_SUM ? acc + v : (op == RED_MIN ? fmin(acc, v) : fmax(acc, v));
  }
  if (op == RED_SUM) acc = block_sum<double, NT>(acc);
  else if (op == RED_MIN) acc = block_min<double, NT>(acc, INFINITY);
  else acc = block_max<double, NT>(acc, -INFINITY);
  if (threadIdx.x == 0) *out = acc;
}

__global__ void k_dinv(Dev S) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < S.nv; v += gridDim.x * blockDim.x) {
    const double* a = S.D + 9 * (int64_t)v;
    double c[9];
    c[0] = a[4] * a[8] - a[5] * a[7];
    c[1] = a[2] * a[7] - a[1] * a[8];
    c[2] = a[1] * a[5] - a[2] * a[4];
    c[3] = a[5] * a[6] - a[3] * a[8];
    c[4] = a[0] * a[8] - a[2] * a[6];
    c[5] = a[2] * a[3] - a[0] * a[5];
    c[6] = a[3] * a[7] - a[4] * a[6];
    c[7] = a[1] * a[6] - a[0] * a[7];
    c[8] = a[0] * a[4] - a[1] * a[3];
    const double det = a[0] * c[0] + a[1] * c[3] + a[2] * c[6];
    const double id = 1.0 / det;
    double* o = S.Dinv + 9 * (int64_t)v;
#pragma unroll
    for (int k = 0; k < 9; ++k) o[k] = c[k] * id;
  }
}

template <typename T>
struct V3 {
  T x, y, z;
};
template <typename T>
__device__ inline V3<T> ldv(const T* __restrict__ p, int64_t i) {
  return V3<T>{p[3 * i], p[3 * i + 1], p[3 * i + 2]};
}
template <typename T>
__device__ inline void stv(T* __restrict__ p, int64_t i, V3<T> v) {
  p[3 * i] = v.x;
  p[3 * i + 1] = v.y;
  p[3 * i + 2] = v.z;
}
template <typename T>
__device__ inline V3<T> addv(V3<T> a, V3<T> b) { return V3<T>{a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename T>
__device__ inline V3<T> axpyv(T s, V3<T> a, V3<T> b) {   // b + s a
  return V3<T>{b.x + s * a.x, b.y + s * a.y, b.z + s * a.z};
}
template <typename T>
__device__ inline T dotv(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T>
__device__ inline V3<T> mv(const T* __restrict__ B, V3<T> v) {
  return V3<T>{B[0] * v.x + B[1] * v.y + B[2] * v.z, B[3] * v.x + B[4] * v.y + B[5] * v.z,
               B[6] * v.x + B[7] * v.y + B[8] * v.z};
}
template <typename T>
__device__ inline V3<T> mtv(const T* __restrict__ B, V3<T> v) {
  return V3<T>{B[0] * v.x + B[3] * v.y + B[6] * v.z, B[1] * v.x + B[4] * v.y + B[7] * v.z,
               B[2] * v.x + B[5] * v.y + B[8] * v.z};
}
template <typename T>
__device__ inline void atomic_addv(T* p, int64_t i, V3<T> v) {
  atomicAdd(p + 3 * i, v.x);
  atomicAdd(p + 3 * i + 1, v.y);
  atomicAdd(p + 3 * i + 2, v.z);
}

template <typename T>
struct OffDiag {
  const int32_t* Lrow;
  const int32_t* Lcol;
  const T* Lval;
  int64_t nL;
  const int32_t* Crow;
  const int32_t* Ccol;
  const T* Cval;
  int64_t nC;
  const int32_t* group;   // non-null: skip blocks whose row and column groups differ (Sec. 4.2.1)
  // 1: difference form -- block (i, j) adds B (v_j - v_i) to row i and
  // B^T (v_i - v_j) to row j, with the diagonal blocks of the system holding
  // G_i = D_i + the sum of row i's off-diagonal blocks (k_diffdiag_rows)
  // instead of D_i
  int diff = 0;
};

// A symmetric block system: diagonal blocks, their inverses, off-diagonal blocks.
template <typename T>
struct Sys {
  const T* D;
  const T* Dinv;
  OffDiag<T> O;
  int nv;
};

template <typename T>
__device__ inline void block_of(const OffDiag<T>& O, int64_t b, int& i, int& j, const T*& B) {
  if (b < O.nL) {
    i = O.Lrow[b];
    j = O.Lcol[b];
    B = O.Lval + 9 * b;
  } else {
    const int64_t c = b - O.nL;
    i = O.Crow[c];
    j = O.Ccol[c];
    B = O.Cval + 9 * c;
  }
}

template <typename T>
__global__ void k_spmv_diag(Sys<T> A, const T* __restrict__ v, T* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.nv; i += gridDim.x * blockDim.x)
    stv(y, i, mv(A.D + 9 * (int64_t)i, ldv(v, i)));
}

template <typename T>
__global__ void k_spmv_offdiag(OffDiag<T> O, const T* __restrict__ v, T* __restrict__ y) {
  const int64_t n = O.nL + O.nC;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n;
       b += (int64_t)gridDim.x * blockDim.x) {
    int i, j;
    const T* B;
    block_of(O, b, i, j, B);
    if (O.group && O.group[i] != O.group[j]) continue;
    if (O.diff) {
      const V3<T> d = axpyv(T(-1), ldv(v, i), ldv(v, j));   // v_j - v_i
      atomic_addv(y, i, mv(B, d));
      atomic_addv(y, j, axpyv(T(-1), mtv(B, d), V3<T>{T(0), T(0), T(0)}));
    } else {
      atomic_addv(y, i, mv(B, ldv(v, j)));
      atomic_addv(y, j, mtv(B, ldv(v, i)));
    }
  }
}

// ---- PCG ------------------------------------------------------------------------------
// Programmatic dependent launch: a PCG-loop kernel lets the next one in the
// stream be scheduled at once, and waits for the previous grid to complete
// (and its writes to be visible) before it reads anything that grid produced.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// last-CTA detection for fused two-level reductions
__device__ inline bool arrive_last(uint32_t* counter) {
  __shared__ bool last;
  __threadfence();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  return last;
}

template <int NT>
__device__ inline double sum_partials(const double* partials, int n) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) acc += ((volatile const double*)partials)[i];
  return block_sum<double, NT>(acc);
}

// r = b - y (y = H x0, or y = null for x0 = 0), z = D^{-1} r; scalars rz, ||r||, ||b||.
// Dot products accumulate in FP64 whatever T is.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_pcg_init(Sys<T> A, const T* __restrict__ b,
                                                 const T* __restrict__ y, T* __restrict__ r,
                                                 T* __restrict__ z, PcgScalars* P,
                                                 double* partials, double tol) {
  double rz = 0.0, rr = 0.0, bb = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < A.nv; i += gridDim.x * NT) {
    const V3<T> bi = ldv(b, i);
    const V3<T> ri = y ? axpyv(T(-1), ldv(y, i), bi) : bi;
    const V3<T> zi = mv(A.Dinv + 9 * (int64_t)i, ri);
    stv(r, i, ri);
    stv(z, i, zi);
    rz += (double)dotv(ri, zi);
    rr += (double)dotv(ri, ri);
    bb += (double)dotv(bi, bi);
  }
  rz = block_sum<double, NT>(rz);
  rr = block_sum<double, NT>(rr);
  bb = block_sum<double, NT>(bb);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = rz;
    partials[gridDim.x + blockIdx.x] = rr;
    partials[2 * gridDim.x + blockIdx.x] = bb;
  }
  if (arrive_last(&P->counter)) {
    const double trz = sum_partials<NT>(partials, gridDim.x);
    const double trr = sum_partials<NT>(partials + gridDim.x, gridDim.x);
    const double tbb = sum_partials<NT>(partials + 2 * gridDim.x, gridDim.x);
    if (threadIdx.x == 0) {
      P->rz = trz;
      P->r0norm = sqrt(trr);
      P->rnorm = P->r0norm;
      P->bnorm = sqrt(tbb);
      P->best = sqrt(fmax(trz, 0.0));
      P->best_it = 0;
      P->it = 0;
      P->tol_abs = tol * P->r0norm;
      P->stagnated = 0;
      P->converged = (P->r0norm == 0.0) ? 1 : 0;
      P->done = P->converged;
      P->beta = 0.0;
      if (!(isfinite(trz) && isfinite(trr))) P->done = 2;
      P->counter = 0;
    }
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_pcg_dir_diag(Sys<T> A, const T* __restrict__ z,
                                                     T* __restrict__ p, T* __restrict__ q,
                                                     PcgScalars* P, double* partials) {
  pdl_enter();
  if (P->done) return;
  const bool first = P->it == 0;
  const T beta = (T)P->beta;
  double pdp = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < A.nv; i += gridDim.x * NT) {
    const V3<T> pi = first ? ldv(z, i) : axpyv(beta, ldv(p, i), ldv(z, i));
    const V3<T> qi = mv(A.D + 9 * (int64_t)i, pi);
    stv(p, i, pi);
    stv(q, i, qi);
    pdp += (double)dotv(pi, qi);
  }
  pdp = block_sum<double, NT>(pdp);
  if (threadIdx.x == 0) partials[blockIdx.x] = pdp;
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_pcg_offdiag(OffDiag<T> O, const T* __restrict__ p,
                                                    T* __restrict__ q, PcgScalars* P,
                                                    double* partials, int n_prev) {
  pdl_enter();
  if (P->done) return;
  const int64_t n = O.nL + O.nC;
  double plp = 0.0;
  for (int64_t b = blockIdx.x * (int64_t)NT + threadIdx.x; b < n; b += (int64_t)gridDim.x * NT) {
    int i, j;
    const T* B;
    block_of(O, b, i, j, B);
    if (O.group && O.group[i] != O.group[j]) continue;
    const V3<T> pj = ldv(p, j), pi = ldv(p, i);
    if (O.diff) {
      const V3<T> d = axpyv(T(-1), pi, pj);   // p_j - p_i
      const V3<T> bd = mv(B, d), btd = mtv(B, d);
      atomic_addv(q, i, bd);
      atomic_addv(q, j, axpyv(T(-1), btd, V3<T>{T(0), T(0), T(0)}));
      plp += (double)dotv(pi, bd) - (double)dotv(pj, btd);
    } else {
      const V3<T> bpj = mv(B, pj);
      atomic_addv(q, i, bpj);
      atomic_addv(q, j, mtv(B, pi));
      plp += 2.0 * (double)dotv(pi, bpj);
    }
  }
  plp = block_sum<double, NT>(plp);
  if (threadIdx.x == 0) partials[n_prev + blockIdx.x] = plp;
  if (arrive_last(&P->counter)) {
    const double pq = sum_partials<NT>(partials, n_prev + gridDim.x);
    if (threadIdx.x == 0) {
      P->pq = pq;
      if (!(pq > 0.0) || !isfinite(pq)) {
        P->done = 3;   // loss of positive definiteness or non-finite
      } else {
        P->alpha = P->rz / pq;
      }
      P->counter = 0;
    }
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_pcg_update(Sys<T> A, T* __restrict__ x,
                                                   const T* __restrict__ p, const T* __restrict__ q,
                                                   T* __restrict__ r, T* __restrict__ z,
                                                   PcgScalars* P, double* partials) {
  pdl_enter();
  if (P->done) return;
  const T alpha = (T)P->alpha;
  double rz = 0.0, rr = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < A.nv; i += gridDim.x * NT) {
    stv(x, i, axpyv(alpha, ldv(p, i), ldv(x, i)));
    const V3<T> ri = axpyv(-alpha, ldv(q, i), ldv(r, i));
    const V3<T> zi = mv(A.Dinv + 9 * (int64_t)i, ri);
    stv(r, i, ri);
    stv(z, i, zi);
    rz += (double)dotv(ri, zi);
    rr += (double)dotv(ri, ri);
  }
  rz = block_sum<double, NT>(rz);
  rr = block_sum<double, NT>(rr);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = rz;
    partials[gridDim.x + blockIdx.x] = rr;
  }
  if (arrive_last(&P->counter)) {
    const double trz = sum_partials<NT>(partials, gridDim.x);
    const double trr = sum_partials<NT>(partials + gridDim.x, gridDim.x);
    if (threadIdx.x == 0) {
      const int it = P->it + 1;
      const double rn = sqrt(trr);
      const double pn = sqrt(fmax(trz, 0.0));   // preconditioned residual norm
      P->it = it;
      P->rnorm = rn;
      if (pn < P->best) {
        P->best = pn;
        P->best_it = it;
      }
      if (!isfinite(rn)) {
        P->done = 2;
      } else if (rn <= P->tol_abs) {
        P->done = 1;
        P->converged = 1;
      } else if (it - P->best_it >= P->window && rn <= P->stall_rel * P->r0norm) {
        P->done = 1;
        P->stagnated = 1;
      } else if (it >= P->max_it) {
        P->done = 1;
      }
      P->beta = trz / P->rz;
      P->rz = trz;
      P->counter = 0;
    }
  }
}

// group_j = floor(log10(e_j)), e_j = sum of node j's three Lambda entries (Sec. 4.2.2)
__global__ void k_groups(const double* __restrict__ lam, int nv, int32_t* __restrict__ grp) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    const double e = lam[3 * v] + lam[3 * v + 1] + lam[3 * v + 2];
    grp[v] = (int32_t)floor(log10(e));
  }
}

// Difference form of the FP32 copy. Every stencil Hessian of H except the
// mass term is translation invariant (elastic energies and contact distances
// depend on position differences only), so the blocks of a row sum to
// m_i/h^2 I, apart from rows that lost blocks to pinned neighbours. Writing
//   (H v)_i = G_i v_i + sum_j B_ij (v_j - v_i),  G_i = D_i + sum_j B_ij
// (sum over row i's off-diagonal blocks, L, C and their transposes), with G_i
// summed in FP64 before its single rounding (it equals m_i/h^2 I to FP64
// rounding in the interior), keeps that invariance exact in FP32: rounding the
// stiff blocks perturbs H v by eps |B| |v_j - v_i| instead of eps |D| |v|, so a
// stiff body's translations, near-null modes of the elastic part that set a
// large share of its condition number, keep their FP32 product equal to H's.
// Its rotations improve less: rounding the FP32 vector itself perturbs each
// vertex by eps |v_i|, which grows with the distance from the axis.
__global__ void k_diffdiag_rows(OffDiag<double> O, double* __restrict__ G) {
  const int64_t n = O.nL + O.nC;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n;
       b += (int64_t)gridDim.x * blockDim.x) {
    int i, j;
    const double* B;
    block_of(O, b, i, j, B);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        atomicAdd(G + 9 * (int64_t)i + 3 * r + c, B[3 * r + c]);   // B in row i
        atomicAdd(G + 9 * (int64_t)j + 3 * r + c, B[3 * c + r]);   // B^T in row j
      }
  }
}

template <typename T>
__global__ void k_convert(int64_t n, const double* __restrict__ a, T* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (T)a[i];
}
// x += s * (double)e ; also r = 0 for the next residual pass
__global__ void k_refine_update(int64_t n, double s, const float* __restrict__ e, double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] += s * (double)e[i];
}
// partial sums of e . r (FP32 e, FP64 r) in FP64
template <int NT>
__global__ void __launch_bounds__(NT) k_dot_fd(int64_t n, const float* __restrict__ e,
                                               const double* __restrict__ r, double* partials) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT)
    acc += (double)e[i] * r[i];
  acc = block_sum<double, NT>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}
// r32 = (float)(r * s)
__global__ void k_scale_to_f32(int64_t n, double s, const double* __restrict__ r, float* __restrict__ o) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    o[i] = (float)(s * r[i]);
}
__global__ void k_sub(int64_t n, const double* __restrict__ b, const double* __restrict__ y,
                      double* __restrict__ r) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - y[i];
}

Sys<double> sys64(Scene& S) {
  Sys<double> A;
  A.D = S.d.D;
  A.Dinv = S.d.Dinv;
  A.O = OffDiag<double>{S.d.L_row, S.d.L_col, S.d.Lval, S.d.nnzL, S.C_row.as<int32_t>(),
                        S.C_col.as<int32_t>(), S.C_val.as<double>(), S.nnzC, nullptr};
  A.nv = S.d.nv;
  return A;
}
Sys<float> sys32(Scene& S) {
  Sys<float> A;
  A.D = S.D32;
  A.Dinv = S.Dinv32;
  A.O = OffDiag<float>{S.d.L_row, S.d.L_col, S.Lval32, S.d.nnzL, S.C_row.as<int32_t>(),
                       S.C_col.as<int32_t>(), S.C_val32.as<float>(), S.nnzC, nullptr,
                       S.f32_form == BAL_MIXED_OP_DIFFERENCE ? 1 : 0};
  A.nv = S.d.nv;
  return A;
}

// launch with programmatic stream serialisation (the kernel calls pdl_enter)
template <typename... K, typename... Args>
cudaError_t launch_pdl(void (*kernel)(K...), int grid, int block, cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename T>
bal_status spmv_t(const Sys<T>& A, const T* v, T* y, cudaStream_t st) {
  k_spmv_diag<T><<<grid_for(A.nv), kThreads, 0, st>>>(A, v, y);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  if (A.O.nL + A.O.nC > 0) {
    k_spmv_offdiag<T><<<grid_for(A.O.nL + A.O.nC, kThreads, kNumSM * 16), kThreads, 0, st>>>(A.O, v, y);
    ::bal::note_launch();
    BAL_LAUNCH_CHECK();
  }
  return BAL_OK;
}

// Block-Jacobi PCG on system A from x (x0 = 0 if y0 is null, else y0 = A x0).
template <typename T>
bal_status pcg_core(Scene& S, const Sys<T>& A, const T* b, const T* y0, T* x, T* r, T* z, T* p,
                    T* q, double tol, int max_it, int window, PcgScalars* hout, cudaStream_t st) {
  constexpr int NT = kRedThreads;
  const int G = kRedBlocks;
  PcgScalars init{};
  init.max_it = max_it;
  init.window = window > 0 ? window : (1 << 30);
  init.stall_rel = S.prm.pcg_stall_forcing > 0 ? S.prm.pcg_stall_forcing : INFINITY;
  BAL_CUDA(cudaMemcpyAsync(S.pcg, &init, sizeof(init), cudaMemcpyHostToDevice, st));
  k_pcg_init<T, NT><<<G, NT, 0, st>>>(A, b, y0, r, z, S.pcg, S.partials, tol);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  PcgScalars h{};
  const int chunk = Scene::kTimedPerChunk;
  int launched = 0, timed = 0;
  for (;;) {
    BAL_CUDA(cudaMemcpyAsync(&h, S.pcg, sizeof(h), cudaMemcpyDeviceToHost, st));
    BAL_CUDA(cudaStreamSynchronize(st));
    BAL_TRY(kt_collect(S, timed));
    timed = 0;
    if (h.done || launched >= max_it) break;
    const int n = std::min(chunk, max_it - launched);
    for (int k = 0; k < n; ++k) {
      BAL_CUDA(launch_pdl(k_pcg_dir_diag<T, NT>, G, NT, st, A, (const T*)z, p, q, S.pcg, S.partials));
      ::bal::note_launch();
      // one off-diagonal product per chunk is timed: an event between two
      // launches ends their programmatic overlap
      if (k == 0) kt_before(S, 0, st);
      BAL_CUDA(launch_pdl(k_pcg_offdiag<T, NT>, G, NT, st, A.O, (const T*)p, q, S.pcg, S.partials, G));
      if (k == 0) {
        kt_after(S, 0, st);
        ++timed;
      }
      ::bal::note_launch();
      BAL_CUDA(launch_pdl(k_pcg_update<T, NT>, G, NT, st, A, x, (const T*)p, (const T*)q, r, z, S.pcg,
                          S.partials));
      ::bal::note_launch();
    }
    BAL_LAUNCH_CHECK();
    launched += n;
  }
  *hout = h;
  if (h.done == 2 || h.done == 3) {
    set_error("pcg: %s at iteration %d", h.done == 2 ? "non-finite residual" : "p^T H p <= 0", h.it);
    return BAL_ERR_NAN;
  }
  return BAL_OK;
}

// ---- two-level additive preconditioner (App. A, comparison only) ------------------
// M^{-1} = D^{-1} + sum_g B_g^T (B_g H B_g^T)^{-1} B_g over groups g of
// kAddGroup consecutive vertices (27x27 blocks), each inverse formed once per
// assembly by Gauss-Jordan elimination (H is SPD, so no pivoting).
constexpr int kAddGroup = 9;
constexpr int kAddN = 3 * kAddGroup;   // 27
constexpr int kAddWarps = 4;

// one warp per group: gather B_g H B_g^T, invert in shared memory, store
__global__ void __launch_bounds__(32 * kAddWarps) k_add_setup(Dev S, const int32_t* __restrict__ crow,
                                                              const int32_t* __restrict__ ccol,
                                                              const double* __restrict__ cval, int64_t nC,
                                                              int ngroups, double* __restrict__ inv) {
  __shared__ double Msh[kAddWarps][kAddN][kAddN + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = blockIdx.x * kAddWarps + w;
  if (g >= ngroups) return;
  double(*M)[kAddN + 1] = Msh[w];
  const int v0 = g * kAddGroup, ng = min(kAddGroup, S.nv - v0);
  for (int e = lane; e < kAddN * kAddN; e += 32) M[e / kAddN][e % kAddN] = 0.0;
  __syncwarp();
  for (int e = lane; e < kAddN; e += 32)
    if (e >= 3 * ng) M[e][e] = 1.0;   // padding rows of the last group: identity
  for (int e = lane; e < 9 * ng; e += 32) {
    const int a = e / 9, k = e % 9;
    M[3 * a + k / 3][3 * a + k % 3] = S.D[9 * (int64_t)(v0 + a) + k];
  }
  __syncwarp();
  if (lane < ng) {   // lane = local row: static lower blocks inside the group, both ways
    const int v = v0 + lane;
    for (int32_t sl = S.L_row_ptr[v]; sl < S.L_row_ptr[v + 1]; ++sl) {
      const int j = S.L_col[sl] - v0;
      if (j < 0 || j >= ng) continue;
      const double* B = S.Lval + 9 * (int64_t)sl;
      for (int k = 0; k < 9; ++k) {
        M[3 * lane + k / 3][3 * j + k % 3] = B[k];
        M[3 * j + k % 3][3 * lane + k / 3] = B[k];
      }
    }
    int lo = 0, hi = (int)nC;   // contact lower blocks of row v (sorted by row, col)
    while (lo < hi) {
      const int m = (lo + hi) >> 1;
      if (crow[m] < v) lo = m + 1;
      else hi = m;
    }
    for (int c = lo; c < nC && crow[c] == v; ++c) {
      const int j = ccol[c] - v0;
      if (j < 0 || j >= ng) continue;
      const double* B = cval + 9 * (int64_t)c;
      for (int k = 0; k < 9; ++k) {
        M[3 * lane + k / 3][3 * j + k % 3] += B[k];
        M[3 * j + k % 3][3 * lane + k / 3] += B[k];
      }
    }
  }
  __syncwarp();
  // in-place Gauss-Jordan inversion
  for (int k = 0; k < kAddN; ++k) {
    const double piv = M[k][k];
    __syncwarp();
    if (lane < kAddN) M[k][lane] = (lane == k ? 1.0 : M[k][lane]) / piv;
    __syncwarp();
    for (int i = 0; i < kAddN; ++i) {
      if (i == k) continue;
      const double f = M[i][k];
      __syncwarp();
      if (lane < kAddN) M[i][lane] = (lane == k ? 0.0 : M[i][lane]) - f * M[k][lane];
      __syncwarp();
    }
  }
  for (int e = lane; e < kAddN * kAddN; e += 32)
    inv[(int64_t)g * kAddN * kAddN + e] = M[e / kAddN][e % kAddN];
}

// x += alpha p, r -= alpha q; partial sums of r.r (at rr_partials)
template <int NT>
__global__ void __launch_bounds__(NT) k_add_update(int nv, double* __restrict__ x, const double* __restrict__ p,
                                                   const double* __restrict__ q, double* __restrict__ r,
                                                   PcgScalars* P, double* rr_partials) {
  if (P->done) return;
  const double alpha = P->alpha;
  double rr = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < 3 * nv; i += gridDim.x * NT) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    rr += ri * ri;
  }
  rr = block_sum<double, NT>(rr);
  if (threadIdx.x == 0) rr_partials[blockIdx.x] = rr;
}

// z = D^{-1} r + sum_g inv_g r_g, one warp per group; partial sums of r.z.
// init: sets rz, best and the first direction state; otherwise also sums the
// r.r partials of k_add_update and decides convergence, stagnation and beta.
template <int NT>
__global__ void __launch_bounds__(NT) k_add_apply(Dev S, int ngroups, const double* __restrict__ inv,
                                                  const double* __restrict__ r, double* __restrict__ z,
                                                  PcgScalars* P, double* partials, const double* rr_partials,
                                                  int n_rr, int init) {
  if (!init && P->done) return;
  constexpr int W = NT / 32;
  const int lane = threadIdx.x & 31;
  double rz = 0.0;
  for (int g = blockIdx.x * W + (threadIdx.x >> 5); g < ngroups; g += gridDim.x * W) {
    const int v0 = g * kAddGroup, ng = min(kAddGroup, S.nv - v0);
    const bool row = lane < 3 * ng;
    const double rl = row ? r[3 * (int64_t)v0 + lane] : 0.0;
    const double* Ig = inv + (int64_t)g * kAddN * kAddN + (row ? lane : 0) * kAddN;
    double acc = 0.0;
    for (int j = 0; j < kAddN; ++j) {   // every lane shuffles; rows past the group ignore the sum
      const double rj = __shfl_sync(0xffffffffu, rl, j);
      if (row) acc += Ig[j] * rj;
    }
    if (row) {
      // block-Jacobi part of the same row
      const int a = lane / 3, c = lane % 3;
      const double* Di = S.Dinv + 9 * (int64_t)(v0 + a) + 3 * c;
      const double* rv = r + 3 * (int64_t)(v0 + a);
      acc += Di[0] * rv[0] + Di[1] * rv[1] + Di[2] * rv[2];
      z[3 * (int64_t)v0 + lane] = acc;
      rz += rl * acc;
    }
  }
  rz = block_sum<double, NT>(rz);
  if (threadIdx.x == 0) partials[blockIdx.x] = rz;
  if (arrive_last(&P->counter)) {
    const double trz = sum_partials<NT>(partials, gridDim.x);
    const double trr = init ? 0.0 : sum_partials<NT>(rr_partials, n_rr);
    if (threadIdx.x == 0) {
      if (init) {
        P->rz = trz;
        P->best = sqrt(fmax(trz, 0.0));
        if (!isfinite(trz)) P->done = 2;
      } else {
        const int it = P->it + 1;
        const double rn = sqrt(trr);
        const double pn = sqrt(fmax(trz, 0.0));
        P->it = it;
        P->rnorm = rn;
        if (pn < P->best) {
          P->best = pn;
          P->best_it = it;
        }
        if (!isfinite(rn)) P->done = 2;
        else if (rn <= P->tol_abs) {
          P->done = 1;
          P->converged = 1;
        } else if (it - P->best_it >= P->window && rn <= P->stall_rel * P->r0norm) {
          P->done = 1;
          P->stagnated = 1;
        } else if (it >= P->max_it) {
          P->done = 1;
        }
        P->beta = trz / P->rz;
        P->rz = trz;
      }
      P->counter = 0;
    }
  }
}

}  // namespace

bal_status finish_reduce_offset(Scene& S, int offset, int n, int slot, RedOp op, cudaStream_t st) {
  k_finish<256><<<1, 256, 0, st>>>(S.partials + offset, n, S.scal + slot, (int)op);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  return BAL_OK;
}

template <typename T>
static bal_status compact_t(Scene& S, const T* in, const uint8_t* flag, int64_t n, T* out,
                            int64_t* nsel, cudaStream_t st) {
  int64_t* dn = reinterpret_cast<int64_t*>(S.scal + 62);
  size_t tmp = 0;
  BAL_CUDA(cub::DeviceSelect::Flagged(nullptr, tmp, in, flag, out, dn, n, st));
  BAL_TRY(buf_reserve(S.cub_tmp, tmp));
  BAL_CUDA(cub::DeviceSelect::Flagged(S.cub_tmp.p, tmp, in, flag, out, dn, n, st));
  BAL_CUDA(cudaMemcpyAsync(nsel, dn, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  return BAL_OK;
}
bal_status compact_u64(Scene& S, const uint64_t* in, const uint8_t* flag, int64_t n, uint64_t* out,
                       int64_t* nsel, cudaStream_t st) {
  if (n <= 0) {
    *nsel = 0;
    return BAL_OK;
  }
  return compact_t(S, in, flag, n, out, nsel, st);
}
bal_status compact_f64(Scene& S, const double* in, const uint8_t* flag, int64_t n, double* out,
                       int64_t* nsel, cudaStream_t st) {
  if (n <= 0) {
    *nsel = 0;
    return BAL_OK;
  }
  return compact_t(S, in, flag, n, out, nsel, st);
}

bal_status launch_dinv(Scene& S, cudaStream_t st) {
  k_dinv<<<grid_for(S.d.nv), kThreads, 0, st>>>(S.d);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  return BAL_OK;
}

bal_status make_f32_copy(Scene& S, cudaStream_t st) {
  const int64_t n9 = 9 * (int64_t)S.d.nv;
  if (S.prm.mixed_operator == BAL_MIXED_OP_DIFFERENCE) {
    BAL_TRY(buf_reserve(S.f32_S, sizeof(double) * n9));
    double* G = S.f32_S.as<double>();
    BAL_CUDA(cudaMemcpyAsync(G, S.d.D, sizeof(double) * n9, cudaMemcpyDeviceToDevice, st));
    const Sys<double> A = sys64(S);
    if (A.O.nL + A.O.nC > 0) {
      k_diffdiag_rows<<<grid_for(A.O.nL + A.O.nC, kThreads, kNumSM * 16), kThreads, 0, st>>>(A.O, G);
      ::bal::note_launch();
    }
    k_convert<float><<<grid_for(n9), kThreads, 0, st>>>(n9, G, S.D32);
    ::bal::note_launch();
  } else {
    k_convert<float><<<grid_for(n9), kThreads, 0, st>>>(n9, S.d.D, S.D32);
    ::bal::note_launch();
  }
  S.f32_form = S.prm.mixed_operator;
  k_convert<float><<<grid_for(n9), kThreads, 0, st>>>(n9, S.d.Dinv, S.Dinv32);
  ::bal::note_launch();
  if (S.d.nnzL) {
    k_convert<float><<<grid_for(9 * S.d.nnzL), kThreads, 0, st>>>(9 * S.d.nnzL, S.d.Lval, S.Lval32);
    ::bal::note_launch();
  }
  BAL_TRY(buf_reserve(S.C_val32, sizeof(float) * 9 * (S.nnzC + 1)));
  if (S.nnzC) {
    k_convert<float><<<grid_for(9 * S.nnzC), kThreads, 0, st>>>(9 * S.nnzC, S.C_val.as<double>(),
                                                                 S.C_val32.as<float>());
    ::bal::note_launch();
  }
  BAL_LAUNCH_CHECK();
  return BAL_OK;
}

bal_status spmv(Scene& S, const double* v, double* y, cudaStream_t st) {
  return spmv_t(sys64(S), v, y, st);
}

bal_status spmv32(Scene& S, const float* v, float* y, cudaStream_t st) {
  return spmv_t(sys32(S), v, y, st);
}

static bal_status true_residual(Scene& S, const double* b, const double* x, double* rn, double* bn,
                                cudaStream_t st) {
  BAL_TRY(spmv(S, x, S.pcg_q, st));
  BAL_TRY(launch_residual_norm(S, b, S.pcg_q, st));
  double res[2];
  BAL_CUDA(cudaMemcpyAsync(res, S.scal + 8, sizeof(res), cudaMemcpyDeviceToHost, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  *rn = sqrt(res[0]);
  *bn = sqrt(res[1]);
  return BAL_OK;
}

bal_status residual_fp64(Scene& S, const double* b, const double* x, double* r, double* rn,
                         double* bn, cudaStream_t st) {
  const int64_t n3 = 3 * (int64_t)S.d.nv;
  BAL_TRY(spmv(S, x, S.pcg_q, st));
  k_sub<<<grid_for(n3), kThreads, 0, st>>>(n3, b, S.pcg_q, r);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  BAL_TRY(launch_residual_norm(S, b, S.pcg_q, st));
  double res[2];
  BAL_CUDA(cudaMemcpyAsync(res, S.scal + 8, sizeof(res), cudaMemcpyDeviceToHost, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  *rn = sqrt(res[0]);
  *bn = sqrt(res[1]);
  return BAL_OK;
}

// e . r in FP64 for the FP32 correction e and an FP64 residual r (host value)
static bal_status dot_fd(Scene& S, int64_t n3, const float* e, const double* r, double* out, cudaStream_t st) {
  k_dot_fd<kRedThreads><<<kRedBlocks, kRedThreads, 0, st>>>(n3, e, r, S.partials);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  BAL_TRY(finish_reduce(S, kRedBlocks, 30, RED_SUM, st));
  BAL_CUDA(cudaMemcpyAsync(out, S.scal + 30, sizeof(double), cudaMemcpyDeviceToHost, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  return BAL_OK;
}

// FP32 inner PCG on the FP32 copy of H, FP64 outer residual and correction
// (iterative refinement): r = b - H x (FP64), solve H e = r/||r|| in FP32 to
// mixed_inner_tol, trial x + d with d = ||r|| e, repeat until ||r|| <= tol
// ||r_0||. A pass is kept if it lowers the FP64 quadratic model f(x) =
// x^T H x / 2 - b^T x -- the energy-norm error, which CG reduces
// monotonically even while ||r||_2 rises -- or the FP64 residual. The change
// of f is formed from the correction and the two residuals,
// f(x + d) - f(x) = -d.(r + r_new) / 2 (r_new = r - H d), so it carries no
// cancellation against f itself and stays meaningful down to the tolerance.
// A pass that lowers neither is rolled back and ends the solve. On exit
// without convergence x is the iterate with the smallest FP64 residual seen.
static bal_status pcg_mixed(Scene& S, const double* b, double* x, double tol, int max_it,
                            bal_solve_info* info, cudaStream_t st) {
  if (!S.f32_valid || S.f32_form != S.prm.mixed_operator) {
    BAL_TRY(make_f32_copy(S, st));
    S.f32_valid = true;
  }
  const int64_t n3 = 3 * (int64_t)S.d.nv;
  double* xtrial = S.pcg_p;   // FP64 work vectors the FP64 solvers own; free here
  double* xbest = S.pcg_z;
  double rn, bn;
  BAL_TRY(residual_fp64(S, b, x, S.pcg_r, &rn, &bn, st));
  const double r0 = rn;
  double best_rn = rn;
  bool best_is_x = true;
  int total = 0, passes = 0;
  bool converged = rn <= tol * r0 || rn == 0.0;
  const Sys<float> A = sys32(S);
  while (!converged && passes < S.prm.mixed_max_refine && total < max_it) {
    k_scale_to_f32<<<grid_for(n3), kThreads, 0, st>>>(n3, 1.0 / rn, S.pcg_r, S.b32);
    ::bal::note_launch();
    BAL_CUDA(cudaMemsetAsync(S.x32, 0, sizeof(float) * n3, st));
    BAL_LAUNCH_CHECK();
    PcgScalars h;
    const int inner = std::min(S.prm.mixed_inner_max, max_it - total);
    const double itol = std::max(S.prm.mixed_inner_tol, 0.5 * tol * r0 / rn);
    const bal_status ist = pcg_core<float>(S, A, S.b32, nullptr, S.x32, S.r32, S.z32, S.p32, S.q32, itol,
                                           inner, S.prm.pcg_stall_window, &h, st);
    // p^T H p <= 0 in FP32 (the FP32 copy of an ill-conditioned H loses
    // definiteness in rounding) ends the inner solve: the iterate before it
    // stands and the FP64 tests below decide; a non-finite residual is an error
    if (ist != BAL_OK && h.done != 3) return ist;
    total += h.it;
    passes += 1;
    if (h.it == 0) break;
    double er, er_new;   // e . r before and after the pass (d = rn e)
    BAL_TRY(dot_fd(S, n3, S.x32, S.pcg_r, &er, st));
    BAL_CUDA(cudaMemcpyAsync(xtrial, x, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
    k_refine_update<<<grid_for(n3), kThreads, 0, st>>>(n3, rn, S.x32, xtrial);
    ::bal::note_launch();
    BAL_LAUNCH_CHECK();
    double rn_new, bn2;
    BAL_TRY(residual_fp64(S, b, xtrial, S.pcg_r, &rn_new, &bn2, st));
    if (!std::isfinite(rn_new)) {
      set_error("mixed pcg: non-finite residual after refinement pass %d", passes);
      return BAL_ERR_NAN;
    }
    BAL_TRY(dot_fd(S, n3, S.x32, S.pcg_r, &er_new, st));
    const double df = -0.5 * rn * (er + er_new);   // f(x + d) - f(x)
    if (!(df < 0.0) && !(rn_new < rn)) {
      // neither the energy-norm error (f) nor the FP64 residual fell: roll the
      // pass back (x and its residual norm stay those of the previous pass;
      // S.pcg_r is not used after the loop)
      break;
    }
    if (best_is_x) {   // x is about to change and holds the smallest residual so far
      BAL_CUDA(cudaMemcpyAsync(xbest, x, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
      best_is_x = false;
    }
    BAL_CUDA(cudaMemcpyAsync(x, xtrial, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
    rn = rn_new;
    if (rn <= best_rn) {
      best_rn = rn;
      best_is_x = true;
    }
    converged = rn <= tol * r0;
  }
  if (!converged && !best_is_x) {
    BAL_CUDA(cudaMemcpyAsync(x, xbest, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
    rn = best_rn;
  }
  if (info) {
    info->iters = total;
    info->rel_residual = bn > 0 ? rn / bn : rn;
    info->rel_residual_r0 = r0 > 0 ? rn / r0 : rn;
    info->stagnated = converged ? 0 : 1;
    info->converged = converged ? 1 : 0;
    info->refine_passes = passes;
    info->warm_iters = 0;
    info->n_groups = 0;
    info->negative_curvature = 0;
    info->precision_used = S.prm.precision == BAL_PREC_FP32 ? BAL_PREC_FP32 : BAL_PREC_MIXED;
  }
  return BAL_OK;
}

// PCG with the two-level additive preconditioner (App. A), FP64; the
// direction, off-diagonal and scalar kernels are those of the block-Jacobi
// solver, the update splits into the vector update and the preconditioner.
static bal_status pcg_additive(Scene& S, const double* b, double* x, double tol, int max_it,
                               bal_solve_info* info, cudaStream_t st) {
  const int nv = S.d.nv;
  const int ngroups = (nv + kAddGroup - 1) / kAddGroup;
  BAL_TRY(buf_reserve(S.add_inv, sizeof(double) * kAddN * kAddN * (size_t)ngroups));
  k_add_setup<<<(ngroups + kAddWarps - 1) / kAddWarps, 32 * kAddWarps, 0, st>>>(
      S.d, S.C_row.as<int32_t>(), S.C_col.as<int32_t>(), S.C_val.as<double>(), S.nnzC, ngroups,
      S.add_inv.as<double>());
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  constexpr int NT = kRedThreads;
  const int G = kRedBlocks;
  const int Ga = std::min((ngroups + NT / 32 - 1) / (NT / 32), kMaxPartials / 2);
  double* rr_part = S.partials + kMaxPartials / 2;
  const Sys<double> A = sys64(S);
  BAL_TRY(spmv(S, x, S.pcg_q, st));
  PcgScalars init{};
  init.max_it = max_it;
  init.window = S.prm.pcg_stall_window > 0 ? S.prm.pcg_stall_window : (1 << 30);
  init.stall_rel = S.prm.pcg_stall_forcing > 0 ? S.prm.pcg_stall_forcing : INFINITY;
  BAL_CUDA(cudaMemcpyAsync(S.pcg, &init, sizeof(init), cudaMemcpyHostToDevice, st));
  k_pcg_init<double, NT><<<G, NT, 0, st>>>(A, b, S.pcg_q, S.pcg_r, S.pcg_z, S.pcg, S.partials, tol);
  ::bal::note_launch();
  k_add_apply<NT><<<Ga, NT, 0, st>>>(S.d, ngroups, S.add_inv.as<double>(), S.pcg_r, S.pcg_z, S.pcg,
                                     S.partials, rr_part, G, 1);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  PcgScalars h{};
  int launched = 0;
  for (;;) {
    BAL_CUDA(cudaMemcpyAsync(&h, S.pcg, sizeof(h), cudaMemcpyDeviceToHost, st));
    BAL_CUDA(cudaStreamSynchronize(st));
    if (h.done || launched >= max_it) break;
    const int n = std::min(16, max_it - launched);
    for (int k = 0; k < n; ++k) {
      k_pcg_dir_diag<double, NT><<<G, NT, 0, st>>>(A, S.pcg_z, S.pcg_p, S.pcg_q, S.pcg, S.partials);
      k_pcg_offdiag<double, NT><<<G, NT, 0, st>>>(A.O, S.pcg_p, S.pcg_q, S.pcg, S.partials, G);
      k_add_update<NT><<<G, NT, 0, st>>>(nv, x, S.pcg_p, S.pcg_q, S.pcg_r, S.pcg, rr_part);
      k_add_apply<NT><<<Ga, NT, 0, st>>>(S.d, ngroups, S.add_inv.as<double>(), S.pcg_r, S.pcg_z, S.pcg,
                                         S.partials, rr_part, G, 0);
      ::bal::note_launch(4);
    }
    BAL_LAUNCH_CHECK();
    launched += n;
  }
  if (h.done == 2 || h.done == 3) {
    set_error("additive pcg: %s at iteration %d", h.done == 2 ? "non-finite residual" : "p^T H p <= 0", h.it);
    return BAL_ERR_NAN;
  }
  if (info) {
    info->iters = h.it;
    info->stagnated = h.stagnated;
    info->converged = h.converged;
    info->refine_passes = 0;
    info->negative_curvature = 0;
    info->precision_used = BAL_PREC_FP64;
    double rn, bn;
    BAL_TRY(true_residual(S, b, x, &rn, &bn, st));
    info->rel_residual = bn > 0 ? rn / bn : rn;
    info->rel_residual_r0 = h.r0norm > 0 ? rn / h.r0norm : rn;
  }
  return BAL_OK;
}

// Stiffness-grouped warm start (Sec. 4.2.2): block-Jacobi PCG on H_dom, the
// Hessian without the blocks that couple different stiffness groups (a masked
// SpMV), run to warm_tol or warm_max_iter from x; its result is x.
static bal_status warm_start(Scene& S, const double* b, double* x, int* iters, int* ngroups,
                             cudaStream_t st) {
  k_groups<<<grid_for(S.d.nv), kThreads, 0, st>>>(S.d.Lambda, S.d.nv, S.group);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  Sys<double> A = sys64(S);
  A.O.group = S.group;
  BAL_TRY(spmv_t(A, x, S.pcg_q, st));
  PcgScalars h;
  BAL_TRY(pcg_core<double>(S, A, b, S.pcg_q, x, S.pcg_r, S.pcg_z, S.pcg_p, S.pcg_q, S.prm.warm_tol,
                           S.prm.warm_max_iter, 1 << 30, &h, st));
  *iters = h.it;
  // number of distinct groups (min/max span) for the report
  std::vector<int32_t> g(S.d.nv);
  BAL_CUDA(cudaMemcpyAsync(g.data(), S.group, sizeof(int32_t) * S.d.nv, cudaMemcpyDeviceToHost, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  std::vector<int32_t> u(g);
  std::sort(u.begin(), u.end());
  *ngroups = (int)(std::unique(u.begin(), u.end()) - u.begin());
  return BAL_OK;
}

bal_status pcg_solve(Scene& S, const double* b, double* x, double tol, int max_it,
                     bal_solve_info* info, cudaStream_t st) {
  int witers = 0, ngroups = 0;
  if (S.prm.precond == BAL_PRECOND_BJ_WARMSTART)
    BAL_TRY(warm_start(S, b, x, &witers, &ngroups, st));
  if (S.prm.precond == BAL_PRECOND_ADDITIVE) {   // FP64 whatever the precision setting
    // as for block-Jacobi below: the FP64 residual decides, with restarts from
    // it while the recursion has drifted below tolerance
    bal_solve_info ai{};
    BAL_TRY(pcg_additive(S, b, x, tol, max_it, &ai, st));
    const double r0 = ai.rel_residual_r0 > 0 ? ai.rel_residual / ai.rel_residual_r0 : 0.0;   // ||r_0|| / ||b||
    int total = ai.iters, restarts = 0;
    double prev = INFINITY;
    while (ai.converged && ai.rel_residual > tol * r0 && restarts < S.prm.mixed_max_refine && total < max_it &&
           ai.rel_residual < 0.99 * prev) {
      prev = ai.rel_residual;
      ++restarts;
      bal_solve_info bi{};
      BAL_TRY(pcg_additive(S, b, x, tol * r0 / ai.rel_residual, max_it - total, &bi, st));
      total += bi.iters;
      ai.converged = bi.converged;
      ai.stagnated = bi.stagnated;
      ai.rel_residual = bi.rel_residual;
    }
    ai.converged = ai.converged && ai.rel_residual <= tol * r0;
    if (info) {
      *info = ai;
      info->iters = total;
      info->refine_passes = restarts;
      info->rel_residual_r0 = r0 > 0 ? ai.rel_residual / r0 : ai.rel_residual;
      info->warm_iters = 0;
      info->n_groups = 0;
    }
    return BAL_OK;
  }
  if (S.prm.precision == BAL_PREC_DF64) {
    BAL_TRY(pcg_df64(S, b, x, tol, max_it, info, st));
    if (info) {
      info->warm_iters = witers;
      info->n_groups = ngroups;
    }
    return BAL_OK;
  }
  if (S.prm.precision == BAL_PREC_MIXED || S.prm.precision == BAL_PREC_FP32) {
    BAL_TRY(pcg_mixed(S, b, x, tol, max_it, info, st));
    if (info) {
      info->warm_iters = witers;
      info->n_groups = ngroups;
    }
    return BAL_OK;
  }
  BAL_TRY(spmv(S, x, S.pcg_q, st));
  PcgScalars h;
  BAL_TRY(pcg_core<double>(S, sys64(S), b, S.pcg_q, x, S.pcg_r, S.pcg_z, S.pcg_p, S.pcg_q, tol,
                           max_it, S.prm.pcg_stall_window, &h, st));
  // On a very ill-conditioned system the recursive residual of FP64 CG drifts
  // from b - H x (the gap reaches a few tolerances at kappa ~ 1e8). When the
  // recursion reports convergence, the FP64 residual decides: CG restarts from
  // it while it is above tol ||r_0|| (at most mixed_max_refine restarts, within
  // max_it iterations in total); a restart that does not lower the FP64
  // residual by 1% (the rounding floor of H x) ends the solve unconverged.
  const double r0 = h.r0norm;
  int total = h.it, restarts = 0;
  bool converged = h.converged != 0, stagnated = h.stagnated != 0, have_true = false;
  double rn = 0.0, bn = 0.0, prev = INFINITY;
  while (converged) {
    BAL_TRY(true_residual(S, b, x, &rn, &bn, st));   // leaves H x in S.pcg_q
    have_true = true;
    if (rn <= tol * r0 || restarts >= S.prm.mixed_max_refine || total >= max_it || !(rn < 0.99 * prev)) {
      converged = rn <= tol * r0;
      break;
    }
    prev = rn;
    ++restarts;
    BAL_TRY(pcg_core<double>(S, sys64(S), b, S.pcg_q, x, S.pcg_r, S.pcg_z, S.pcg_p, S.pcg_q, tol * r0 / rn,
                             max_it - total, S.prm.pcg_stall_window, &h, st));
    total += h.it;
    converged = h.converged != 0;
    stagnated = h.stagnated != 0;
    have_true = false;
  }
  if (info) {
    info->iters = total;
    info->stagnated = stagnated ? 1 : 0;
    info->converged = converged ? 1 : 0;
    info->refine_passes = restarts;
    info->warm_iters = witers;
    info->n_groups = ngroups;
    info->negative_curvature = 0;
    info->precision_used = BAL_PREC_FP64;
    if (!have_true) BAL_TRY(true_residual(S, b, x, &rn, &bn, st));
    info->rel_residual = bn > 0 ? rn / bn : rn;
    info->rel_residual_r0 = r0 > 0 ? rn / r0 : rn;
  }
  return BAL_OK;
}

namespace {
template <int NT>
__global__ void __launch_bounds__(NT) k_resid(Dev S, const double* __restrict__ b,
                                              const double* __restrict__ y, double* partials) {
  double rr = 0.0, bb = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < S.nv; i += gridDim.x * NT) {
    const d3 bi = ld3(b, i);
    const d3 ri = bi - ld3(y, i);
    rr += dot(ri, ri);
    bb += dot(bi, bi);
  }
  rr = block_sum<double, NT>(rr);
  bb = block_sum<double, NT>(bb);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = rr;
    partials[gridDim.x + blockIdx.x] = bb;
  }
}
}  // namespace

bal_status launch_residual_norm(Scene& S, const double* b, const double* y, cudaStream_t st) {
  k_resid<256><<<kRedBlocks, 256, 0, st>>>(S.d, b, y, S.partials);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  BAL_TRY(finish_reduce_offset(S, 0, kRedBlocks, 8, RED_SUM, st));
  BAL_TRY(finish_reduce_offset(S, kRedBlocks, kRedBlocks, 9, RED_SUM, st));
  return BAL_OK;
}

}  // namespace bal
