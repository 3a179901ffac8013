// bal_pcg_solve_noalloc: block-Jacobi PCG on a caller-provided symmetric block
// matrix whose working memory is a fixed, file-scope device array instead of
// allocations.
//
// Who needs it: callers that must not allocate GPU memory during their run --
// code that runs while a memory pool or an allocator lock is held by the host
// application, real-time loops that forbid allocation after start-up, and
// plug-ins whose host owns every device allocation. bal_pcg_solve works on a
// scene created by bal_create_scene (which allocates); this entry point needs
// nothing but the caller's input and output buffers.
//
// The scratch (PCG vectors r, z, p, q, block inverses, partial sums and the
// solver scalars) lives in g_scratch below. Every GPU that loads the library
// holds this array until the process exits. The host-side name g_scratch is not
// a device address, so each device's address is looked up once with
// cudaGetSymbolAddress (with that device current) on the first call made on it;
// make that first call before any stream capture. All calls share the array:
// calls that overlap on the GPU (different streams, threads or processes using
// the same context) race on it and must be serialised by the caller.
#include <mutex>

#include "common.cuh"

namespace bal {
namespace {

constexpr int kNaMaxVerts = BAL_NOALLOC_MAX_VERTS;
constexpr int kNaBlocks = 2 * kNumSM;
constexpr int kNaThreads = 256;

struct NaScalars {
  double rz, pq, alpha, beta, r0norm, rnorm, bnorm, best, tol_abs;
  int32_t it, best_it, done, stagnated, converged, max_it, window, pad;
  uint32_t counter, pad2;
};

// layout of the scratch array (in doubles)
constexpr size_t kVec = 3 * (size_t)kNaMaxVerts;
constexpr size_t kOffR = 0, kOffZ = kVec, kOffP = 2 * kVec, kOffQ = 3 * kVec;
constexpr size_t kOffDinv = 4 * kVec;                       // 9 per vertex
constexpr size_t kOffPart = kOffDinv + 9 * (size_t)kNaMaxVerts;
constexpr size_t kOffScal = kOffPart + 4 * kNaBlocks;
constexpr size_t kScratchDoubles = kOffScal + 32;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_addr[64] = {nullptr};

struct NaMat {
  const double* D;
  const int32_t* rows;
  const int32_t* cols;
  const double* vals;
  int64_t nnz;
  int nv;
};

__device__ inline void na_mv(const double* B, const double* v, double o[3], bool tr) {
  for (int i = 0; i < 3; ++i)
    o[i] = tr ? B[i] * v[0] + B[3 + i] * v[1] + B[6 + i] * v[2]
              : B[3 * i] * v[0] + B[3 * i + 1] * v[1] + B[3 * i + 2] * v[2];
}

__device__ inline bool na_last(uint32_t* counter) {
  __shared__ bool last;
  __threadfence();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  return last;
}

__device__ inline double na_sum(const double* part, int n) {
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += kNaThreads) a += ((volatile const double*)part)[i];
  return block_sum<double, kNaThreads>(a);
}

// D^{-1} per vertex, r = b - H x0 is formed by the caller's x0 = sol: first q = H x0
__global__ void k_na_dinv_diag(NaMat A, double* S, const double* __restrict__ x) {
  double* Dinv = S + kOffDinv;
  double* q = S + kOffQ;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < A.nv; v += gridDim.x * blockDim.x) {
    const double* a = A.D + 9 * (int64_t)v;
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
    const double id = 1.0 / (a[0] * c[0] + a[1] * c[3] + a[2] * c[6]);
    for (int k = 0; k < 9; ++k) Dinv[9 * (int64_t)v + k] = c[k] * id;
    double o[3];
    na_mv(a, x + 3 * (int64_t)v, o, false);
    for (int k = 0; k < 3; ++k) q[3 * (int64_t)v + k] = o[k];
  }
}

__global__ void k_na_offdiag_apply(NaMat A, const double* __restrict__ v, double* y) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < A.nnz;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int i = A.rows[b], j = A.cols[b];
    const double* B = A.vals + 9 * b;
    double o[3];
    na_mv(B, v + 3 * (int64_t)j, o, false);
    for (int k = 0; k < 3; ++k) atomicAdd(y + 3 * (int64_t)i + k, o[k]);
    na_mv(B, v + 3 * (int64_t)i, o, true);
    for (int k = 0; k < 3; ++k) atomicAdd(y + 3 * (int64_t)j + k, o[k]);
  }
}

__global__ void __launch_bounds__(kNaThreads) k_na_init(NaMat A, double* S, const double* __restrict__ b,
                                                        double tol) {
  double *r = S + kOffR, *z = S + kOffZ, *q = S + kOffQ, *Dinv = S + kOffDinv, *part = S + kOffPart;
  NaScalars* P = reinterpret_cast<NaScalars*>(S + kOffScal);
  double rz = 0.0, rr = 0.0, bb = 0.0;
  for (int i = blockIdx.x * kNaThreads + threadIdx.x; i < A.nv; i += gridDim.x * kNaThreads) {
    double ri[3], zi[3];
    for (int k = 0; k < 3; ++k) {
      ri[k] = b[3 * (int64_t)i + k] - q[3 * (int64_t)i + k];
      bb += b[3 * (int64_t)i + k] * b[3 * (int64_t)i + k];
    }
    na_mv(Dinv + 9 * (int64_t)i, ri, zi, false);
    for (int k = 0; k < 3; ++k) {
      r[3 * (int64_t)i + k] = ri[k];
      z[3 * (int64_t)i + k] = zi[k];
      rz += ri[k] * zi[k];
      rr += ri[k] * ri[k];
    }
  }
  rz = block_sum<double, kNaThreads>(rz);
  rr = block_sum<double, kNaThreads>(rr);
  bb = block_sum<double, kNaThreads>(bb);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = rz;
    part[gridDim.x + blockIdx.x] = rr;
    part[2 * gridDim.x + blockIdx.x] = bb;
  }
  if (na_last(&P->counter)) {
    const double trz = na_sum(part, gridDim.x), trr = na_sum(part + gridDim.x, gridDim.x);
    const double tbb = na_sum(part + 2 * gridDim.x, gridDim.x);
    if (threadIdx.x == 0) {
      P->rz = trz;
      P->r0norm = P->rnorm = sqrt(trr);
      P->best = sqrt(fmax(trz, 0.0));   // stagnation is judged on the preconditioned norm
      P->bnorm = sqrt(tbb);
      P->tol_abs = tol * P->r0norm;
      P->it = P->best_it = 0;
      P->converged = P->r0norm == 0.0 ? 1 : 0;
      P->done = P->converged;
      if (!(isfinite(trz) && isfinite(trr))) P->done = 2;
      P->counter = 0;
    }
  }
}

__global__ void __launch_bounds__(kNaThreads) k_na_dir(NaMat A, double* S) {
  NaScalars* P = reinterpret_cast<NaScalars*>(S + kOffScal);
  if (P->done) return;
  double *z = S + kOffZ, *p = S + kOffP, *q = S + kOffQ, *part = S + kOffPart;
  const bool first = P->it == 0;
  const double beta = P->beta;
  double pdp = 0.0;
  for (int i = blockIdx.x * kNaThreads + threadIdx.x; i < A.nv; i += gridDim.x * kNaThreads) {
    double pi[3], qi[3];
    for (int k = 0; k < 3; ++k)
      pi[k] = first ? z[3 * (int64_t)i + k] : z[3 * (int64_t)i + k] + beta * p[3 * (int64_t)i + k];
    na_mv(A.D + 9 * (int64_t)i, pi, qi, false);
    for (int k = 0; k < 3; ++k) {
      p[3 * (int64_t)i + k] = pi[k];
      q[3 * (int64_t)i + k] = qi[k];
      pdp += pi[k] * qi[k];
    }
  }
  pdp = block_sum<double, kNaThreads>(pdp);
  if (threadIdx.x == 0) part[blockIdx.x] = pdp;
}

__global__ void __launch_bounds__(kNaThreads) k_na_off(NaMat A, double* S) {
  NaScalars* P = reinterpret_cast<NaScalars*>(S + kOffScal);
  if (P->done) return;
  double *p = S + kOffP, *q = S + kOffQ, *part = S + kOffPart;
  double plp = 0.0;
  for (int64_t b = blockIdx.x * (int64_t)kNaThreads + threadIdx.x; b < A.nnz;
       b += (int64_t)gridDim.x * kNaThreads) {
    const int i = A.rows[b], j = A.cols[b];
    const double* B = A.vals + 9 * b;
    double o[3];
    na_mv(B, p + 3 * (int64_t)j, o, false);
    for (int k = 0; k < 3; ++k) {
      atomicAdd(q + 3 * (int64_t)i + k, o[k]);
      plp += 2.0 * p[3 * (int64_t)i + k] * o[k];
    }
    na_mv(B, p + 3 * (int64_t)i, o, true);
    for (int k = 0; k < 3; ++k) atomicAdd(q + 3 * (int64_t)j + k, o[k]);
  }
  plp = block_sum<double, kNaThreads>(plp);
  if (threadIdx.x == 0) part[gridDim.x + blockIdx.x] = plp;
  if (na_last(&P->counter)) {
    const double pq = na_sum(part, 2 * gridDim.x);
    if (threadIdx.x == 0) {
      P->pq = pq;
      if (!(pq > 0.0) || !isfinite(pq)) P->done = 3;
      else P->alpha = P->rz / pq;
      P->counter = 0;
    }
  }
}

__global__ void __launch_bounds__(kNaThreads) k_na_update(NaMat A, double* S, double* __restrict__ x) {
  NaScalars* P = reinterpret_cast<NaScalars*>(S + kOffScal);
  if (P->done) return;
  double *r = S + kOffR, *z = S + kOffZ, *p = S + kOffP, *q = S + kOffQ, *Dinv = S + kOffDinv,
         *part = S + kOffPart;
  const double alpha = P->alpha;
  double rz = 0.0, rr = 0.0;
  for (int i = blockIdx.x * kNaThreads + threadIdx.x; i < A.nv; i += gridDim.x * kNaThreads) {
    double ri[3], zi[3];
    for (int k = 0; k < 3; ++k) {
      x[3 * (int64_t)i + k] += alpha * p[3 * (int64_t)i + k];
      ri[k] = r[3 * (int64_t)i + k] - alpha * q[3 * (int64_t)i + k];
    }
    na_mv(Dinv + 9 * (int64_t)i, ri, zi, false);
    for (int k = 0; k < 3; ++k) {
      r[3 * (int64_t)i + k] = ri[k];
      z[3 * (int64_t)i + k] = zi[k];
      rz += ri[k] * zi[k];
      rr += ri[k] * ri[k];
    }
  }
  rz = block_sum<double, kNaThreads>(rz);
  rr = block_sum<double, kNaThreads>(rr);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = rz;
    part[gridDim.x + blockIdx.x] = rr;
  }
  if (na_last(&P->counter)) {
    const double trz = na_sum(part, gridDim.x), trr = na_sum(part + gridDim.x, gridDim.x);
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
      if (!isfinite(rn)) P->done = 2;
      else if (rn <= P->tol_abs) P->done = 1, P->converged = 1;
      else if (it - P->best_it >= P->window) P->done = 1, P->stagnated = 1;
      else if (it >= P->max_it) P->done = 1;
      P->beta = trz / P->rz;
      P->rz = trz;
      P->counter = 0;
    }
  }
}

// ||b - H x||^2 and ||b||^2 into the first two scalar slots after the solve
__global__ void __launch_bounds__(kNaThreads) k_na_resid(NaMat A, double* S, const double* __restrict__ b) {
  double *q = S + kOffQ, *part = S + kOffPart;
  NaScalars* P = reinterpret_cast<NaScalars*>(S + kOffScal);
  double rr = 0.0, bb = 0.0;
  for (int i = blockIdx.x * kNaThreads + threadIdx.x; i < 3 * A.nv; i += gridDim.x * kNaThreads) {
    const double d = b[i] - q[i];
    rr += d * d;
    bb += b[i] * b[i];
  }
  rr = block_sum<double, kNaThreads>(rr);
  bb = block_sum<double, kNaThreads>(bb);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = rr;
    part[gridDim.x + blockIdx.x] = bb;
  }
  if (na_last(&P->counter)) {
    const double a = na_sum(part, gridDim.x), c = na_sum(part + gridDim.x, gridDim.x);
    if (threadIdx.x == 0) {
      P->rnorm = sqrt(a);
      P->bnorm = sqrt(c);
      P->counter = 0;
    }
  }
}

__global__ void k_na_diag_apply(NaMat A, const double* __restrict__ v, double* y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.nv; i += gridDim.x * blockDim.x) {
    double o[3];
    na_mv(A.D + 9 * (int64_t)i, v + 3 * (int64_t)i, o, false);
    for (int k = 0; k < 3; ++k) y[3 * (int64_t)i + k] = o[k];
  }
}

bal_status scratch_address(double** out) {
  int dev = 0;
  BAL_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("bal_pcg_solve_noalloc: device index %d out of range", dev);
    return BAL_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_scratch)", __FILE__, __LINE__);
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return BAL_OK;
}

}  // namespace
}  // namespace bal

using namespace bal;

extern "C" bal_status bal_pcg_solve_noalloc(int32_t n_verts, const double* D, int64_t nnz,
                                            const int32_t* rows, const int32_t* cols,
                                            const double* vals, const double* rhs, double* sol,
                                            double rel_tol, int32_t max_iter,
                                            bal_solve_info* info, void* stream) {
  if (n_verts <= 0 || n_verts > kNaMaxVerts) {
    set_error("bal_pcg_solve_noalloc: n_verts = %d outside [1, %d] (BAL_NOALLOC_MAX_VERTS)", n_verts,
              kNaMaxVerts);
    return BAL_ERR_ARG;
  }
  if (!D || !rhs || !sol || nnz < 0 || (nnz > 0 && (!rows || !cols || !vals)) || !(rel_tol >= 0) ||
      max_iter < 0) {
    set_error("bal_pcg_solve_noalloc: invalid pointer, nnz, tolerance or iteration cap");
    return BAL_ERR_ARG;
  }
  double* S = nullptr;
  BAL_TRY(scratch_address(&S));
  cudaStream_t st = (cudaStream_t)stream;
  const NaMat A{D, rows, cols, vals, nnz, n_verts};
  const int G = kNaBlocks, NT = kNaThreads;
  NaScalars init{};
  init.max_it = max_iter;
  init.window = 100;
  NaScalars* P = reinterpret_cast<NaScalars*>(S + kOffScal);
  BAL_CUDA(cudaMemcpyAsync(P, &init, sizeof(init), cudaMemcpyHostToDevice, st));
  // q = H sol (diagonal part with D^{-1}, then off-diagonal blocks), r, z, scalars
  k_na_dinv_diag<<<grid_for(n_verts), NT, 0, st>>>(A, S, sol);
  if (nnz > 0) k_na_offdiag_apply<<<grid_for(nnz, NT, kNumSM * 16), NT, 0, st>>>(A, sol, S + kOffQ);
  k_na_init<<<G, NT, 0, st>>>(A, S, rhs, rel_tol);
  BAL_LAUNCH_CHECK();
  NaScalars h{};
  int launched = 0;
  for (;;) {
    BAL_CUDA(cudaMemcpyAsync(&h, P, sizeof(h), cudaMemcpyDeviceToHost, st));
    BAL_CUDA(cudaStreamSynchronize(st));
    if (h.done || launched >= max_iter) break;
    const int n = std::min(16, max_iter - launched);
    for (int k = 0; k < n; ++k) {
      k_na_dir<<<G, NT, 0, st>>>(A, S);
      k_na_off<<<G, NT, 0, st>>>(A, S);
      k_na_update<<<G, NT, 0, st>>>(A, S, sol);
    }
    BAL_LAUNCH_CHECK();
    launched += n;
  }
  if (info) {
    // true residual ||rhs - H sol|| in FP64
    k_na_diag_apply<<<grid_for(n_verts), NT, 0, st>>>(A, sol, S + kOffQ);
    if (nnz > 0) k_na_offdiag_apply<<<grid_for(nnz, NT, kNumSM * 16), NT, 0, st>>>(A, sol, S + kOffQ);
    k_na_resid<<<G, NT, 0, st>>>(A, S, rhs);
    BAL_LAUNCH_CHECK();
    NaScalars f{};
    BAL_CUDA(cudaMemcpyAsync(&f, P, sizeof(f), cudaMemcpyDeviceToHost, st));
    BAL_CUDA(cudaStreamSynchronize(st));
    info->iters = h.it;
    info->rel_residual = f.bnorm > 0 ? f.rnorm / f.bnorm : f.rnorm;
    info->rel_residual_r0 = h.r0norm > 0 ? f.rnorm / h.r0norm : f.rnorm;
    info->stagnated = h.stagnated;
    info->converged = h.converged;
    info->refine_passes = 0;
    info->warm_iters = 0;
    info->n_groups = 0;
  }
  if (h.done == 2 || h.done == 3) {
    set_error("bal_pcg_solve_noalloc: %s at iteration %d",
              h.done == 2 ? "non-finite residual" : "p^T H p <= 0", h.it);
    return BAL_ERR_NAN;
  }
  return BAL_OK;
}
