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
// ||r_0||), stagnation (no new minimum of ||r|| in `window` iterations) and
// beta. Once `done` is set the remaining launches of a chunk return at once, so
// the host only synchronises once per chunk of iterations.
#include <cub/cub.cuh>

#include "scene.cuh"

namespace bal {

namespace {

constexpr int kRedBlocks = 2 * kNumSM;   // CTAs of every fused reduction kernel
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

// ---- contact blocks: heads of equal-key runs, then per-run sums -------------------
__global__ void k_iota(int32_t* a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = (int32_t)i;
}
__global__ void k_heads(const uint64_t* __restrict__ k, int64_t n, int32_t* __restrict__ head) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    head[i] = (k[i] != ~0ull && (i == 0 || k[i] != k[i - 1])) ? 1 : 0;
}
__global__ void k_segsum(const uint64_t* __restrict__ k, const int32_t* __restrict__ idx,
                         const double* __restrict__ vals, const int32_t* __restrict__ head,
                         const int32_t* __restrict__ pos, int64_t n, int32_t* __restrict__ crow,
                         int32_t* __restrict__ ccol, double* __restrict__ cval) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!head[i]) continue;
    const uint64_t key = k[i];
    double acc[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) acc[c] = 0.0;
    for (int64_t j = i; j < n && k[j] == key; ++j) {
      const double* v = vals + 9 * (int64_t)idx[j];
#pragma unroll
      for (int c = 0; c < 9; ++c) acc[c] += v[c];
    }
    const int32_t o = pos[i];
    crow[o] = (int32_t)(key >> 32);
    ccol[o] = (int32_t)(key & 0xffffffffu);
#pragma unroll
    for (int c = 0; c < 9; ++c) cval[9 * (int64_t)o + c] = acc[c];
  }
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

__device__ inline d3 mv(const double* __restrict__ B, d3 v) {
  return d3{B[0] * v.x + B[1] * v.y + B[2] * v.z, B[3] * v.x + B[4] * v.y + B[5] * v.z,
            B[6] * v.x + B[7] * v.y + B[8] * v.z};
}
__device__ inline d3 mtv(const double* __restrict__ B, d3 v) {
  return d3{B[0] * v.x + B[3] * v.y + B[6] * v.z, B[1] * v.x + B[4] * v.y + B[7] * v.z,
            B[2] * v.x + B[5] * v.y + B[8] * v.z};
}

struct OffDiag {
  const int32_t* Lrow;
  const int32_t* Lcol;
  const double* Lval;
  int64_t nL;
  const int32_t* Crow;
  const int32_t* Ccol;
  const double* Cval;
  int64_t nC;
};

__device__ inline void block_of(const OffDiag& O, int64_t b, int& i, int& j, const double*& B) {
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

__global__ void k_spmv_diag(Dev S, const double* __restrict__ v, double* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.nv; i += gridDim.x * blockDim.x)
    st3(y, i, mv(S.D + 9 * (int64_t)i, ld3(v, i)));
}

__global__ void k_spmv_offdiag(OffDiag O, const double* __restrict__ v, double* __restrict__ y) {
  const int64_t n = O.nL + O.nC;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n;
       b += (int64_t)gridDim.x * blockDim.x) {
    int i, j;
    const double* B;
    block_of(O, b, i, j, B);
    atomic_add3(y, i, mv(B, ld3(v, j)));
    atomic_add3(y, j, mtv(B, ld3(v, i)));
  }
}

// ---- PCG ------------------------------------------------------------------------------
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

// r = b - H x (given y = H x), z = D^{-1} r; scalars rz, ||r||, ||b||
template <int NT>
__global__ void __launch_bounds__(NT) k_pcg_init(Dev S, const double* __restrict__ b,
                                                 const double* __restrict__ y, double* __restrict__ r,
                                                 double* __restrict__ z, PcgScalars* P,
                                                 double* partials, double tol) {
  double rz = 0.0, rr = 0.0, bb = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < S.nv; i += gridDim.x * NT) {
    const d3 bi = ld3(b, i);
    const d3 ri = bi - ld3(y, i);
    const d3 zi = mv(S.Dinv + 9 * (int64_t)i, ri);
    st3(r, i, ri);
    st3(z, i, zi);
    rz += dot(ri, zi);
    rr += dot(ri, ri);
    bb += dot(bi, bi);
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
      P->best = P->r0norm;
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

template <int NT>
__global__ void __launch_bounds__(NT) k_pcg_dir_diag(Dev S, const double* __restrict__ z,
                                                     double* __restrict__ p, double* __restrict__ q,
                                                     PcgScalars* P, double* partials) {
  if (P->done) return;
  const double beta = P->it == 0 ? 0.0 : P->beta;
  double pdp = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < S.nv; i += gridDim.x * NT) {
    const d3 pi = P->it == 0 ? ld3(z, i) : ld3(z, i) + beta * ld3(p, i);
    const d3 qi = mv(S.D + 9 * (int64_t)i, pi);
    st3(p, i, pi);
    st3(q, i, qi);
    pdp += dot(pi, qi);
  }
  pdp = block_sum<double, NT>(pdp);
  if (threadIdx.x == 0) partials[blockIdx.x] = pdp;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_pcg_offdiag(OffDiag O, const double* __restrict__ p,
                                                    double* __restrict__ q, PcgScalars* P,
                                                    double* partials, int n_prev) {
  if (P->done) return;
  const int64_t n = O.nL + O.nC;
  double plp = 0.0;
  for (int64_t b = blockIdx.x * (int64_t)NT + threadIdx.x; b < n; b += (int64_t)gridDim.x * NT) {
    int i, j;
    const double* B;
    block_of(O, b, i, j, B);
    const d3 pj = ld3(p, j), pi = ld3(p, i);
    const d3 bpj = mv(B, pj);
    atomic_add3(q, i, bpj);
    atomic_add3(q, j, mtv(B, pi));
    plp += 2.0 * dot(pi, bpj);
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

template <int NT>
__global__ void __launch_bounds__(NT) k_pcg_update(Dev S, double* __restrict__ x,
                                                   const double* __restrict__ p,
                                                   const double* __restrict__ q, double* __restrict__ r,
                                                   double* __restrict__ z, PcgScalars* P,
                                                   double* partials) {
  if (P->done) return;
  const double alpha = P->alpha;
  double rz = 0.0, rr = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < S.nv; i += gridDim.x * NT) {
    st3(x, i, ld3(x, i) + alpha * ld3(p, i));
    const d3 ri = ld3(r, i) - alpha * ld3(q, i);
    const d3 zi = mv(S.Dinv + 9 * (int64_t)i, ri);
    st3(r, i, ri);
    st3(z, i, zi);
    rz += dot(ri, zi);
    rr += dot(ri, ri);
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
      P->it = it;
      P->rnorm = rn;
      if (rn < P->best) {
        P->best = rn;
        P->best_it = it;
      }
      if (!isfinite(rn)) {
        P->done = 2;
      } else if (rn <= P->tol_abs) {
        P->done = 1;
        P->converged = 1;
      } else if (it - P->best_it >= P->window) {
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

OffDiag offdiag_of(Scene& S) {
  OffDiag O;
  O.Lrow = S.d.L_row;
  O.Lcol = S.d.L_col;
  O.Lval = S.d.Lval;
  O.nL = S.d.nnzL;
  O.Crow = S.C_row.as<int32_t>();
  O.Ccol = S.C_col.as<int32_t>();
  O.Cval = S.C_val.as<double>();
  O.nC = S.nnzC;
  return O;
}

}  // namespace

bal_status finish_reduce_offset(Scene& S, int offset, int n, int slot, RedOp op, cudaStream_t st) {
  k_finish<256><<<1, 256, 0, st>>>(S.partials + offset, n, S.scal + slot, (int)op);
  BAL_LAUNCH_CHECK();
  return BAL_OK;
}

bal_status contact_blocks_reduce(Scene& S, int64_t n_emit, cudaStream_t st) {
  S.nnzC = 0;
  if (n_emit <= 0) return BAL_OK;
  BAL_TRY(buf_reserve(S.emit_keys_alt, sizeof(uint64_t) * n_emit));
  BAL_TRY(buf_reserve(S.emit_idx, sizeof(int32_t) * n_emit));
  BAL_TRY(buf_reserve(S.emit_idx_alt, sizeof(int32_t) * n_emit));
  BAL_TRY(buf_reserve(S.seg_head, sizeof(int32_t) * (n_emit + 1)));
  BAL_TRY(buf_reserve(S.seg_pos, sizeof(int32_t) * (n_emit + 1)));
  k_iota<<<grid_for(n_emit), kThreads, 0, st>>>(S.emit_idx.as<int32_t>(), n_emit);
  BAL_LAUNCH_CHECK();
  cub::DoubleBuffer<uint64_t> dk(S.emit_keys.as<uint64_t>(), S.emit_keys_alt.as<uint64_t>());
  cub::DoubleBuffer<int32_t> dv(S.emit_idx.as<int32_t>(), S.emit_idx_alt.as<int32_t>());
  size_t tmp = 0;
  BAL_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp, dk, dv, n_emit, 0, 64, st));
  BAL_TRY(buf_reserve(S.cub_tmp, tmp));
  BAL_CUDA(cub::DeviceRadixSort::SortPairs(S.cub_tmp.p, tmp, dk, dv, n_emit, 0, 64, st));
  int32_t* head = S.seg_head.as<int32_t>();
  int32_t* pos = S.seg_pos.as<int32_t>();
  k_heads<<<grid_for(n_emit), kThreads, 0, st>>>(dk.Current(), n_emit, head);
  BAL_LAUNCH_CHECK();
  BAL_CUDA(cudaMemsetAsync(head + n_emit, 0, sizeof(int32_t), st));
  tmp = 0;
  BAL_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp, head, pos, n_emit + 1, st));
  BAL_TRY(buf_reserve(S.cub_tmp, tmp));
  BAL_CUDA(cub::DeviceScan::ExclusiveSum(S.cub_tmp.p, tmp, head, pos, n_emit + 1, st));
  int32_t nC = 0;
  BAL_CUDA(cudaMemcpyAsync(&nC, pos + n_emit, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  BAL_TRY(buf_reserve(S.C_row, sizeof(int32_t) * (nC + 1)));
  BAL_TRY(buf_reserve(S.C_col, sizeof(int32_t) * (nC + 1)));
  BAL_TRY(buf_reserve(S.C_val, sizeof(double) * 9 * (nC + 1)));
  k_segsum<<<grid_for(n_emit), kThreads, 0, st>>>(dk.Current(), dv.Current(), S.emit_vals.as<double>(),
                                                 head, pos, n_emit, S.C_row.as<int32_t>(),
                                                 S.C_col.as<int32_t>(), S.C_val.as<double>());
  BAL_LAUNCH_CHECK();
  S.nnzC = nC;
  return BAL_OK;
}

bal_status launch_dinv(Scene& S, cudaStream_t st) {
  k_dinv<<<grid_for(S.d.nv), kThreads, 0, st>>>(S.d);
  BAL_LAUNCH_CHECK();
  return BAL_OK;
}

bal_status spmv(Scene& S, const double* v, double* y, cudaStream_t st) {
  k_spmv_diag<<<grid_for(S.d.nv), kThreads, 0, st>>>(S.d, v, y);
  BAL_LAUNCH_CHECK();
  const OffDiag O = offdiag_of(S);
  if (O.nL + O.nC > 0) {
    k_spmv_offdiag<<<grid_for(O.nL + O.nC, kThreads, kNumSM * 16), kThreads, 0, st>>>(O, v, y);
    BAL_LAUNCH_CHECK();
  }
  return BAL_OK;
}

bal_status pcg_solve(Scene& S, const double* b, double* x, double tol, int max_it,
                     bal_solve_info* info, cudaStream_t st) {
  constexpr int NT = kRedThreads;
  const int G = kRedBlocks;
  double* r = S.pcg_r;
  double* z = S.pcg_z;
  double* p = S.pcg_p;
  double* q = S.pcg_q;
  PcgScalars init{};
  init.max_it = max_it;
  init.window = S.prm.pcg_stall_window > 0 ? S.prm.pcg_stall_window : (1 << 30);
  BAL_CUDA(cudaMemcpyAsync(S.pcg, &init, sizeof(init), cudaMemcpyHostToDevice, st));
  BAL_TRY(spmv(S, x, q, st));
  k_pcg_init<NT><<<G, NT, 0, st>>>(S.d, b, q, r, z, S.pcg, S.partials, tol);
  BAL_LAUNCH_CHECK();
  const OffDiag O = offdiag_of(S);
  PcgScalars h{};
  const int chunk = 16;
  int launched = 0;
  for (;;) {
    BAL_CUDA(cudaMemcpyAsync(&h, S.pcg, sizeof(h), cudaMemcpyDeviceToHost, st));
    BAL_CUDA(cudaStreamSynchronize(st));
    if (h.done || launched >= max_it) break;
    const int n = std::min(chunk, max_it - launched);
    for (int k = 0; k < n; ++k) {
      k_pcg_dir_diag<NT><<<G, NT, 0, st>>>(S.d, z, p, q, S.pcg, S.partials);
      k_pcg_offdiag<NT><<<G, NT, 0, st>>>(O, p, q, S.pcg, S.partials, G);
      k_pcg_update<NT><<<G, NT, 0, st>>>(S.d, x, p, q, r, z, S.pcg, S.partials);
    }
    BAL_LAUNCH_CHECK();
    launched += n;
  }
  if (info) {
    info->iters = h.it;
    info->stagnated = h.stagnated;
    info->converged = h.converged;
    info->refine_passes = 0;
    info->warm_iters = 0;
    info->n_groups = 0;
    // true residual, FP64
    BAL_TRY(spmv(S, x, q, st));
    BAL_TRY(launch_residual_norm(S, b, q, st));
    double res[2];
    BAL_CUDA(cudaMemcpyAsync(res, S.scal + 8, sizeof(res), cudaMemcpyDeviceToHost, st));
    BAL_CUDA(cudaStreamSynchronize(st));
    const double rn = sqrt(res[0]), bn = sqrt(res[1]);
    info->rel_residual = bn > 0 ? rn / bn : rn;
    info->rel_residual_r0 = h.r0norm > 0 ? rn / h.r0norm : rn;
  }
  if (h.done == 2 || h.done == 3) {
    set_error("pcg: %s at iteration %d", h.done == 2 ? "non-finite residual" : "p^T H p <= 0", h.it);
    return BAL_ERR_NAN;
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
  BAL_LAUNCH_CHECK();
  BAL_TRY(finish_reduce_offset(S, 0, kRedBlocks, 8, RED_SUM, st));
  BAL_TRY(finish_reduce_offset(S, kRedBlocks, kRedBlocks, 9, RED_SUM, st));
  return BAL_OK;
}

}  // namespace bal
