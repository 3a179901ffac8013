// Block-Jacobi PCG with double-float recurrences (Sec. 4.2, App. B; the
// precision is this library's choice for B300, whose FP64 pipe runs at ~1/58 of
// its FP32 rate).
//
// The same CG iteration as the FP64 solver in matrix.cu, with H, D^{-1} and the
// vectors held as double-floats (dd.cuh, ~47-bit significand) so that every
// iteration runs in FP32 arithmetic and is bound by memory traffic. FP64
// decides convergence: the initial residual r = b - H x and the final one are
// computed with the FP64 matrix; if the recurrence reports convergence but the
// FP64 residual is still above tolerance, CG restarts from the FP64 residual
// (iterative refinement), at most mixed_max_refine times.
//
// H v keeps the paper's symmetric storage (D, L, C; Sec. 5.1) but evaluates it
// as a gather, one thread per row, with no atomics, so the result is
// deterministic. The static lower blocks sit in a sliced-ELL layout: 32 rows
// per slice, entry k of the 32 rows adjacent in memory and the 9 entries of a
// block 32 values apart, so one warp reads a slice with coalesced loads. Rows
// are given to slice lanes after a stable sort by list length within windows
// of 4096 rows (sliced ELL with a sorting window), which removes most of the
// padding that the alternating neighbour counts of a Kuhn-split lattice leave
// in 32 consecutive rows while keeping each slice's rows close in index. Row i
// sums D_i v_i, its own blocks L_ij v_j, then the transposes L_ki^T v_k of the
// blocks stored in later rows k with column i (the column-side list holds their
// value positions); on a lattice ordering those also lie side by side for 32
// adjacent rows, and their second read is served by L2. Contact blocks are
// applied by extra CTAs of the same launch, eight lanes per contact row, into
// a per-contact-row buffer that the update kernel adds to those rows.
#include <algorithm>
#include <utility>

#include "dd.cuh"
#include "scene.cuh"

namespace bal {

namespace {

constexpr int kDdThreads = 256;
constexpr int kDdWarps = kDdThreads / 32;
constexpr double kDdRange = 1e36;        // entries beyond this stay in the FP64 solver
// padding entries read zero blocks; spreading them over this many chunks keeps
// every slice's padding reads on different L2 lines instead of one hot spot
constexpr int kZeroChunks = 64;
// rows are sorted by list length within windows of this many rows (128 slices)
constexpr int kSellWindow = 4096;
// lanes that share one contact row in the contact CTAs of k_dd_spmv
constexpr int kContactLanes = 8;

struct DDSys {
  const dd* D;            // [ns][9][32]
  const dd* Dinv;         // [ns][9][32]
  const int32_t* offR;    // [ns+1]
  const int32_t* Rcol;    // [offR[ns]]
  const dd* R;            // sliced lower blocks, then one chunk of zero blocks
  const int32_t* offT;    // [ns+1]
  const int32_t* Tpos;    // [offT[ns]]
  const int32_t* Tsrc;    // [offT[ns]]
  const short2* len;      // [ns*32] row-side and column-side list length of each slot's row
  const int32_t* srow;    // [ns*32] row of each slot (-1: none)
  int64_t zero;           // value position of the first chunk of zero blocks
  int nv, ns;
};

struct DDContact {
  const int32_t* rows;    // [n] unique rows
  const int32_t* ptr;     // [n+1]
  const int32_t* ent;     // [2 nC] 2c + (1 if C_c^T is applied)
  const int32_t* src;     // [2 nC] source vertex
  const dd* C;            // [nC][9]
  int n;
};

// entry e of the block at value position b of the sliced storage is b[32 e]
__device__ __forceinline__ dd3 mv_sliced(const dd* __restrict__ b, dd3 v) {
  dd B[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) B[k] = b[32 * k];
  return dd3{dd_fma(B[2], v.z, dd_fma(B[1], v.y, dd_mul(B[0], v.x))),
             dd_fma(B[5], v.z, dd_fma(B[4], v.y, dd_mul(B[3], v.x))),
             dd_fma(B[8], v.z, dd_fma(B[7], v.y, dd_mul(B[6], v.x)))};
}
__device__ __forceinline__ dd3 mtv_sliced(const dd* __restrict__ b, dd3 v) {
  dd B[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) B[k] = b[32 * k];
  return dd3{dd_fma(B[6], v.z, dd_fma(B[3], v.y, dd_mul(B[0], v.x))),
             dd_fma(B[7], v.z, dd_fma(B[4], v.y, dd_mul(B[1], v.x))),
             dd_fma(B[8], v.z, dd_fma(B[5], v.y, dd_mul(B[2], v.x)))};
}
// value position of vertex i's block in a slice-major [ns][9][32] array
__device__ __forceinline__ int64_t slice_base(int i) { return (int64_t)(i >> 5) * 9 * 32 + (i & 31); }

__device__ __forceinline__ void dd3_acc(dd3& a, dd3 b) {
  a.x = dd_add(a.x, b.x);
  a.y = dd_add(a.y, b.y);
  a.z = dd_add(a.z, b.z);
}

// D or D^-1 (FP64, [nv][9]) into the slice-major double-float layout, block i
// at slot slot_of[i] (slot i when slot_of is null)
__global__ void k_dd_slices(int nv, const double* __restrict__ a, dd* __restrict__ out, unsigned int* bad,
                            const int32_t* __restrict__ slot_of) {
  const int64_t n = 9 * (int64_t)nv;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / 9), e = (int)(t % 9);
    const double v = a[t];
    if (!(fabs(v) <= kDdRange)) atomicAdd(bad, 1u);
    out[slice_base(slot_of ? slot_of[i] : i) + 32 * e] = dd_from(v);
  }
}
// L values (FP64, CSR slot order [nL][9]) into their sliced positions
__global__ void k_dd_scatter(int64_t nL, const double* __restrict__ L, const int32_t* __restrict__ pos,
                             dd* __restrict__ R, unsigned int* bad) {
  const int64_t n = 9 * nL;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = t / 9;
    const int e = (int)(t % 9);
    const double v = L[t];
    if (!(fabs(v) <= kDdRange)) atomicAdd(bad, 1u);
    R[(int64_t)pos[s] + 32 * e] = dd_from(v);
  }
}
__global__ void k_to_dd(int64_t n, const double* __restrict__ a, dd* __restrict__ b, unsigned int* bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = a[i];
    if (!(fabs(v) <= kDdRange)) atomicAdd(bad, 1u);
    b[i] = dd_from(v);
  }
}

// directed contact entries keyed for the per-vertex bucket sort: entry 2c
// applies C_c to row C_row[c], entry 2c + 1 applies C_c^T to row C_col[c];
// key = row << 32 | entry, so record index = entry
__global__ void k_crow_keys(const int32_t* __restrict__ crow, const int32_t* __restrict__ ccol, int nC,
                            uint64_t* __restrict__ key) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * nC; e += gridDim.x * blockDim.x) {
    const int c = e >> 1;
    const int32_t r = (e & 1) ? ccol[c] : crow[c];
    key[e] = ((uint64_t)(uint32_t)r << 32) | (uint32_t)e;
  }
}
// flag[v] = 1 where vertex v has contact entries
__global__ void k_crow_flag(const int32_t* __restrict__ len, int nv, int32_t* __restrict__ flag) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x)
    flag[v] = len[v] > 0 ? 1 : 0;
}
// contact row r = rpos[v] of each vertex with entries: rows[r] = v, ptr[r] =
// off[v], crow_of[v] = r (-1 for the others); ptr[number of rows] = n2
__global__ void k_crow_rows(const int32_t* __restrict__ len, const int32_t* __restrict__ off,
                            const int32_t* __restrict__ rpos, int nv, int n2, int32_t* __restrict__ rows,
                            int32_t* __restrict__ ptr, int32_t* __restrict__ crow_of) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    if (len[v] > 0) {
      const int r = rpos[v];
      rows[r] = v;
      ptr[r] = off[v];
      crow_of[v] = r;
    } else {
      crow_of[v] = -1;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ptr[rpos[nv]] = n2;
}
// source vertex of each ordered entry
__global__ void k_crow_src(const int32_t* __restrict__ ent, const int32_t* __restrict__ crow,
                           const int32_t* __restrict__ ccol, int n2, int32_t* __restrict__ src) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += gridDim.x * blockDim.x) {
    const int c = ent[e] >> 1;
    src[e] = (ent[e] & 1) ? crow[c] : ccol[c];
  }
}

// Programmatic dependent launch: a PCG-loop kernel lets the next one in the
// stream be scheduled at once, and waits for the previous grid to complete
// (and its writes to be visible) before it reads anything that grid produced.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ inline bool dd_arrive_last(uint32_t* counter) {
  __shared__ bool last;
  __threadfence();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  return last;
}

template <int NT>
__device__ inline double dd_sum_partials(const double* partials, int n) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) acc += ((volatile const double*)partials)[i];
  return block_sum<double, NT>(acc);
}

__device__ inline void set_alpha(PcgScalars* P, double pq) {
  P->pq = pq;
  if (!(pq > 0.0) || !isfinite(pq)) {
    P->done = 3;   // loss of positive definiteness or non-finite
  } else {
    P->alpha = P->rz / pq;
    const dd a = dd_from(P->alpha);
    P->alpha_hi = a.hi;
    P->alpha_lo = a.lo;
  }
}

__device__ __forceinline__ dd3 dinv_apply(const DDSys& A, int i, dd3 r) {
  return mv_sliced(A.Dinv + slice_base(i), r);
}

// r = s * rf (FP64 residual scaled to unit norm), z = D^{-1} r, x = 0; rz, ||r||.
template <int NT>
__global__ void __launch_bounds__(NT) k_dd_init(DDSys A, const double* __restrict__ rf, double s,
                                                dd* __restrict__ x, dd* __restrict__ r,
                                                dd* __restrict__ z, PcgScalars* P, double* partials,
                                                double tol) {
  dd rz{0.f, 0.f}, rr{0.f, 0.f};
  for (int i = blockIdx.x * NT + threadIdx.x; i < A.nv; i += gridDim.x * NT) {
    const dd3 ri{dd_from(s * rf[3 * (int64_t)i]), dd_from(s * rf[3 * (int64_t)i + 1]),
                 dd_from(s * rf[3 * (int64_t)i + 2])};
    const dd3 zi = dinv_apply(A, i, ri);
    dd3_st(r, i, ri);
    dd3_st(z, i, zi);
    dd3_st(x, i, dd3{dd{0.f, 0.f}, dd{0.f, 0.f}, dd{0.f, 0.f}});
    rz = dd_add(rz, dd3_dot(ri, zi));
    rr = dd_add(rr, dd3_dot(ri, ri));
  }
  rz = dd_block_sum<NT>(rz);
  rr = dd_block_sum<NT>(rr);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = dd_to(rz);
    partials[gridDim.x + blockIdx.x] = dd_to(rr);
  }
  if (dd_arrive_last(&P->counter)) {
    const double trz = dd_sum_partials<NT>(partials, gridDim.x);
    const double trr = dd_sum_partials<NT>(partials + gridDim.x, gridDim.x);
    if (threadIdx.x == 0) {
      P->rz = trz;
      P->r0norm = sqrt(trr);
      P->rnorm = P->r0norm;
      P->bnorm = P->r0norm;
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

// p = z + beta p (p = z on the first iteration)
template <int NT>
__global__ void __launch_bounds__(NT) k_dd_dir(int nv, const dd* __restrict__ z, dd* __restrict__ p,
                                               const PcgScalars* P) {
  pdl_enter();
  if (P->done) return;
  const bool first = P->it == 0;
  const dd beta{P->beta_hi, P->beta_lo};
  for (int i = blockIdx.x * NT + threadIdx.x; i < nv; i += gridDim.x * NT) {
    const dd3 zi = dd3_ld(z, i);
    dd3_st(p, i, first ? zi : dd3_axpy(beta, dd3_ld(p, i), zi));
  }
}

// Contact part of H p for contact rows b, b + nb, ... (CTAs of the SpMV grid
// past the slice CTAs): qc_t = sum of the contact blocks of row rows[t], both
// orientations, applied to p. G lanes share a row: lane j of the group takes
// entries j, j + G, ... and the group's sums are combined by shuffles in a
// fixed order (deterministic). Each warp covers 32 / G consecutive rows and
// iterates while any of them exists, so every lane reaches the shuffles.
// Returns this thread's share of sum_t p_rows[t] . qc_t.
template <int G>
__device__ dd contact_rows(const DDContact& Cr, const dd* __restrict__ p, dd* __restrict__ qc, int b, int nb) {
  static_assert(G >= 1 && G <= 32 && (G & (G - 1)) == 0, "G is a power of two <= 32");
  constexpr int kRowsPerWarp = 32 / G;
  const int lane = threadIdx.x & 31, sub = lane & (G - 1);
  const int64_t warp = (b * (int64_t)kDdThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)nb * kDdThreads) >> 5;
  dd pq{0.f, 0.f};
  for (int64_t t0 = warp * kRowsPerWarp; t0 < Cr.n; t0 += nwarps * kRowsPerWarp) {
    const int64_t t = t0 + lane / G;
    const bool valid = t < Cr.n;
    dd3 acc{dd{0.f, 0.f}, dd{0.f, 0.f}, dd{0.f, 0.f}};
    if (valid) {
      const int e1 = Cr.ptr[t + 1];
      for (int e = Cr.ptr[t] + sub; e < e1; e += G) {
        const int ent = Cr.ent[e];
        const dd* B = Cr.C + 9 * (int64_t)(ent >> 1);
        const dd3 v = dd3_ld(p, Cr.src[e]);
        dd3_acc(acc, (ent & 1) ? dd3_mtv(B, v) : dd3_mv(B, v));
      }
    }
#pragma unroll
    for (int off = G / 2; off >= 1; off >>= 1) {
      dd3 o;
      o.x = dd{__shfl_xor_sync(0xffffffffu, acc.x.hi, off), __shfl_xor_sync(0xffffffffu, acc.x.lo, off)};
      o.y = dd{__shfl_xor_sync(0xffffffffu, acc.y.hi, off), __shfl_xor_sync(0xffffffffu, acc.y.lo, off)};
      o.z = dd{__shfl_xor_sync(0xffffffffu, acc.z.hi, off), __shfl_xor_sync(0xffffffffu, acc.z.lo, off)};
      dd3_acc(acc, o);
    }
    if (valid && sub == 0) {
      dd3_st(qc, (int)t, acc);
      pq = dd_add(pq, dd3_dot(dd3_ld(p, Cr.rows[t]), acc));
    }
  }
  return pq;
}

// q = (D + L + L^T) p over the slices (n_row_ctas CTAs) and the contact part
// per contact row into qc (the remaining CTAs, interleaved with them);
// partial sums of p . Hp; the last CTA to finish sets alpha.
__global__ void __launch_bounds__(kDdThreads) k_dd_spmv(DDSys A, DDContact Cr, int n_row_ctas,
                                                        const dd* __restrict__ p, dd* __restrict__ q,
                                                        dd* __restrict__ qc, PcgScalars* P,
                                                        double* partials) {
  pdl_enter();
  if (P->done) return;
  const int lane = threadIdx.x & 31;
  dd pq{0.f, 0.f};
  // contact CTA j sits at grid position j K + K - 1 (K = grid / contact CTAs),
  // so the contact rows' longer serial chains start throughout the launch and
  // overlap the slice CTAs instead of forming a tail; the other positions are
  // the slice CTAs in order
  const int nc = gridDim.x - n_row_ctas;
  const int K = nc > 0 ? (int)gridDim.x / nc : 1;
  const int bj = blockIdx.x / K, br = blockIdx.x % K;
  if (nc > 0 && br == K - 1 && bj < nc) {
    pq = contact_rows<kContactLanes>(Cr, p, qc, bj, nc);
  } else {
    const int bs = blockIdx.x - (nc > 0 ? min(nc, (int)(blockIdx.x + 1) / K) : 0);
    for (int s = bs * kDdWarps + (threadIdx.x >> 5); s < A.ns; s += n_row_ctas * kDdWarps) {
      const int slot = 32 * s + lane;
      const int i = A.srow[slot];
      const bool own = i >= 0;
      const dd3 pi = own ? dd3_ld(p, i) : dd3{dd{0.f, 0.f}, dd{0.f, 0.f}, dd{0.f, 0.f}};
      dd3 acc = mv_sliced(A.D + slice_base(slot), pi);
      // lanes past their own row-side list length (padding) read a zero chunk,
      // which stays in L2; the column-side padding entries already point at one
      const int lr = A.len[slot].x;
      const int r0 = A.offR[s], r1 = A.offR[s + 1];
#pragma unroll 2
      for (int idx = r0 + lane; idx < r1; idx += 32) {
        const int64_t vb = idx - r0 < 32 * lr ? 9 * (int64_t)(idx - lane) + lane
                                              : A.zero + 288 * (s % kZeroChunks) + lane;
        dd3_acc(acc, mv_sliced(A.R + vb, dd3_ld(p, A.Rcol[idx])));
      }
      const int t1 = A.offT[s + 1];
#pragma unroll 2
      for (int idx = A.offT[s] + lane; idx < t1; idx += 32)
        dd3_acc(acc, mtv_sliced(A.R + A.Tpos[idx], dd3_ld(p, A.Tsrc[idx])));
      if (own) {
        dd3_st(q, i, acc);
        pq = dd_add(pq, dd3_dot(pi, acc));
      }
    }
  }
  pq = dd_block_sum<kDdThreads>(pq);
  if (threadIdx.x == 0) partials[blockIdx.x] = dd_to(pq);
  if (dd_arrive_last(&P->counter)) {
    const double tpq = dd_sum_partials<kDdThreads>(partials, gridDim.x);
    if (threadIdx.x == 0) {
      set_alpha(P, tpq);
      P->counter = 0;
    }
  }
}

// q = (D + L + L^T) p with one CTA per window of W consecutive rows (W a
// multiple of 32; the slot order sorts rows only inside their window): p of
// the window's rows is staged in shared memory; every row-side block L_ij
// adds L_ij p_j to its row and, when row j lies in the same window (j < i <
// window end, so j >= window start suffices), L_ij^T p_i to an FP64 shared
// accumulator of row j; the transposes of blocks stored in later windows come
// through the column-side list. Each row's own sum joins the accumulator, and
// q is written in row order after a CTA barrier. The shared FP64 sums take
// their terms in arrival order (atomics), so this layout is not
// bit-reproducible (it is within FP64 rounding of the gather). Contact CTAs
// as in k_dd_spmv.
__device__ __forceinline__ dd3 ps_ld(const dd* ps, int r) { return dd3{ps[3 * r], ps[3 * r + 1], ps[3 * r + 2]}; }

__global__ void __launch_bounds__(kDdThreads, 3) k_dd_spmv_win(DDSys A, DDContact Cr, int n_row_ctas, int W,
                                                            const dd* __restrict__ p, dd* __restrict__ q,
                                                            dd* __restrict__ qc, PcgScalars* P,
                                                            double* partials) {
  extern __shared__ double smw[];   // [W][3] FP64 sums, then [W][3] double-float p
  pdl_enter();
  if (P->done) return;
  const int lane = threadIdx.x & 31;
  dd pq{0.f, 0.f};
  const int nc = gridDim.x - n_row_ctas;
  const int K = nc > 0 ? (int)gridDim.x / nc : 1;
  const int bj = blockIdx.x / K, br = blockIdx.x % K;
  if (nc > 0 && br == K - 1 && bj < nc) {
    pq = contact_rows<kContactLanes>(Cr, p, qc, bj, nc);
  } else {
    const int w = blockIdx.x - (nc > 0 ? min(nc, (int)(blockIdx.x + 1) / K) : 0);
    const int w0 = w * W, w1 = min(A.nv, w0 + W), nw = w1 - w0;
    double* acc = smw;
    dd* ps = reinterpret_cast<dd*>(smw + 3 * W);
    for (int r = threadIdx.x; r < nw; r += kDdThreads) {
      const dd3 v = dd3_ld(p, w0 + r);
      ps[3 * r] = v.x;
      ps[3 * r + 1] = v.y;
      ps[3 * r + 2] = v.z;
      acc[3 * r] = acc[3 * r + 1] = acc[3 * r + 2] = 0.0;
    }
    __syncthreads();
    const int s0 = w0 >> 5, s1 = (w1 + 31) >> 5;
    for (int s = s0 + (threadIdx.x >> 5); s < s1; s += kDdWarps) {
      const int slot = 32 * s + lane;
      const int i = A.srow[slot];
      const bool own = i >= 0;
      const dd3 pi = own ? ps_ld(ps, i - w0) : dd3{dd{0.f, 0.f}, dd{0.f, 0.f}, dd{0.f, 0.f}};
      dd3 a = mv_sliced(A.D + slice_base(slot), pi);
      const int lr = A.len[slot].x;
      const int r0 = A.offR[s], r1 = A.offR[s + 1];
#pragma unroll 2
      for (int idx = r0 + lane; idx < r1; idx += 32) {
        const bool real = idx - r0 < 32 * lr;
        const int64_t vb = real ? 9 * (int64_t)(idx - lane) + lane : A.zero + 288 * (s % kZeroChunks) + lane;
        const int j = A.Rcol[idx];
        const dd* b = A.R + vb;
        dd B[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) B[k] = b[32 * k];
        const bool inw = j >= w0;
        const dd3 pj = inw ? ps_ld(ps, j - w0) : dd3_ld(p, j);
        a.x = dd_add(a.x, dd_fma(B[2], pj.z, dd_fma(B[1], pj.y, dd_mul(B[0], pj.x))));
        a.y = dd_add(a.y, dd_fma(B[5], pj.z, dd_fma(B[4], pj.y, dd_mul(B[3], pj.x))));
        a.z = dd_add(a.z, dd_fma(B[8], pj.z, dd_fma(B[7], pj.y, dd_mul(B[6], pj.x))));
        if (real && inw) {   // L_ij^T p_i into row j's shared sum
          double* aj = acc + 3 * (j - w0);
          atomicAdd(aj, dd_to(dd_fma(B[6], pi.z, dd_fma(B[3], pi.y, dd_mul(B[0], pi.x)))));
          atomicAdd(aj + 1, dd_to(dd_fma(B[7], pi.z, dd_fma(B[4], pi.y, dd_mul(B[1], pi.x)))));
          atomicAdd(aj + 2, dd_to(dd_fma(B[8], pi.z, dd_fma(B[5], pi.y, dd_mul(B[2], pi.x)))));
        }
      }
      const int t1 = A.offT[s + 1];
#pragma unroll 2
      for (int idx = A.offT[s] + lane; idx < t1; idx += 32)
        dd3_acc(a, mtv_sliced(A.R + A.Tpos[idx], dd3_ld(p, A.Tsrc[idx])));
      if (own) {
        double* ai = acc + 3 * (i - w0);
        atomicAdd(ai, dd_to(a.x));
        atomicAdd(ai + 1, dd_to(a.y));
        atomicAdd(ai + 2, dd_to(a.z));
      }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nw; r += kDdThreads) {
      const dd3 qv{dd_from(acc[3 * r]), dd_from(acc[3 * r + 1]), dd_from(acc[3 * r + 2])};
      dd3_st(q, w0 + r, qv);
      pq = dd_add(pq, dd3_dot(ps_ld(ps, r), qv));
    }
  }
  pq = dd_block_sum<kDdThreads>(pq);
  if (threadIdx.x == 0) partials[blockIdx.x] = dd_to(pq);
  if (dd_arrive_last(&P->counter)) {
    const double tpq = dd_sum_partials<kDdThreads>(partials, gridDim.x);
    if (threadIdx.x == 0) {
      set_alpha(P, tpq);
      P->counter = 0;
    }
  }
}

// x += alpha p, r -= alpha q, z = D^{-1} r; rz, ||r||; convergence, stagnation, beta
template <int NT>
__global__ void __launch_bounds__(NT) k_dd_update(DDSys A, dd* __restrict__ x, const dd* __restrict__ p,
                                                  const dd* __restrict__ q, const int32_t* __restrict__ crow_of,
                                                  const dd* __restrict__ qc, dd* __restrict__ r,
                                                  dd* __restrict__ z, PcgScalars* P, double* partials) {
  pdl_enter();
  if (P->done) return;
  const dd alpha{P->alpha_hi, P->alpha_lo};
  const dd malpha = dd_neg(alpha);
  dd rz{0.f, 0.f}, rr{0.f, 0.f};
  // unrolled over two vertices per thread (on large meshes the grid is halved):
  // more independent loads in flight
#pragma unroll 2
  for (int i = blockIdx.x * NT + threadIdx.x; i < A.nv; i += gridDim.x * NT) {
    dd3_st(x, i, dd3_axpy(alpha, dd3_ld(p, i), dd3_ld(x, i)));
    dd3 qi = dd3_ld(q, i);
    if (crow_of) {   // H p of a contact row: slice part + contact part
      const int c = crow_of[i];
      if (c >= 0) dd3_acc(qi, dd3_ld(qc, c));
    }
    const dd3 ri = dd3_axpy(malpha, qi, dd3_ld(r, i));
    const dd3 zi = dinv_apply(A, i, ri);
    dd3_st(r, i, ri);
    dd3_st(z, i, zi);
    rz = dd_add(rz, dd3_dot(ri, zi));
    rr = dd_add(rr, dd3_dot(ri, ri));
  }
  rz = dd_block_sum<NT>(rz);
  rr = dd_block_sum<NT>(rr);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = dd_to(rz);
    partials[gridDim.x + blockIdx.x] = dd_to(rr);
  }
  if (dd_arrive_last(&P->counter)) {
    const double trz = dd_sum_partials<NT>(partials, gridDim.x);
    const double trr = dd_sum_partials<NT>(partials + gridDim.x, gridDim.x);
    if (threadIdx.x == 0) {
      const int it = P->it + 1;
      const double rn = sqrt(trr);
      const double pn = sqrt(fmax(trz, 0.0));
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
      const dd b = dd_from(P->beta);
      P->beta_hi = b.hi;
      P->beta_lo = b.lo;
      P->rz = trz;
      P->counter = 0;
    }
  }
}

// x += s * e (FP64 += double-float)
__global__ void k_dd_accumulate(int64_t n, double s, const dd* __restrict__ e, double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += s * dd_to(e[i]);
}

// Sliced layout of the static lower blocks from the host CSR copy (once per
// layout). win = 0: sorting windows of kSellWindow rows and full column-side
// lists; win > 0: sorting windows of win rows (the windows of k_dd_spmv_win)
// and column-side lists holding only the blocks stored in other windows.
bal_status build_sell(Scene& S, int win) {
  const int nv = S.d.nv;
  const int sw = win > 0 ? win : kSellWindow;
  const int64_t nL = S.d.nnzL;
  const int ns = (nv + 31) / 32;
  const std::vector<int32_t>& rp = S.row_ptr_h;
  const std::vector<int32_t>& col = S.col_h;
  // column lists (ascending row) of the lower blocks; with windows, only the
  // blocks whose row lies in another window than their column
  auto listed = [&](int r, int c) { return win <= 0 || r / win != c / win; };
  std::vector<int32_t> cp(nv + 1, 0);
  for (int r = 0; r < nv; ++r)
    for (int32_t s = rp[r]; s < rp[r + 1]; ++s)
      if (listed(r, col[s])) cp[col[s] + 1]++;
  for (int v = 0; v < nv; ++v) cp[v + 1] += cp[v];
  const int64_t nList = cp[nv];
  std::vector<int32_t> cslot(nList > 0 ? nList : 1), crow(nList > 0 ? nList : 1);
  {
    std::vector<int32_t> fill(cp.begin(), cp.end() - 1);
    for (int r = 0; r < nv; ++r)
      for (int32_t s = rp[r]; s < rp[r + 1]; ++s) {
        if (!listed(r, col[s])) continue;
        const int32_t e = fill[col[s]]++;
        cslot[e] = s;
        crow[e] = r;
      }
  }
  // slot order: within each window of kSellWindow rows, rows sorted by
  // row-side list length, then column-side length (descending, stable), so the
  // 32 rows of a slice have near-equal lists and the slices carry little
  // padding (on a Kuhn-split lattice the lower-neighbour counts alternate
  // between 3 and 7 from one row to the next)
  std::vector<int32_t> srow((size_t)ns * 32, -1), slot_of(nv);
  for (int w0 = 0; w0 < nv; w0 += sw) {
    const int w1 = std::min(nv, w0 + sw);
    std::vector<int32_t> rows(w1 - w0);
    for (int i = w0; i < w1; ++i) rows[i - w0] = i;
    std::stable_sort(rows.begin(), rows.end(), [&](int32_t a, int32_t b) {
      const int la = rp[a + 1] - rp[a], lb = rp[b + 1] - rp[b];
      if (la != lb) return la > lb;
      return cp[a + 1] - cp[a] > cp[b + 1] - cp[b];
    });
    for (int k = 0; k < w1 - w0; ++k) {
      srow[w0 + k] = rows[k];
      slot_of[rows[k]] = w0 + k;
    }
  }
  std::vector<int32_t> offR(ns + 1, 0), offT(ns + 1, 0);
  for (int s = 0; s < ns; ++s) {
    int lr = 0, lt = 0;
    for (int l = 0; l < 32; ++l) {
      const int i = srow[32 * s + l];
      if (i < 0) break;
      lr = std::max(lr, rp[i + 1] - rp[i]);
      lt = std::max(lt, cp[i + 1] - cp[i]);
    }
    if ((int64_t)offR[s] + 32 * (int64_t)lr > (INT32_MAX / 9 - 32 * kZeroChunks) ||
        (int64_t)offT[s] + 32 * (int64_t)lt > INT32_MAX) {
      set_error("df64 pcg: sliced storage exceeds 32-bit positions");
      return BAL_ERR_CAPACITY;
    }
    offR[s + 1] = offR[s] + 32 * lr;
    offT[s + 1] = offT[s] + 32 * lt;
  }
  const int64_t nR = offR[ns], nT = offT[ns];
  const int32_t zero = 9 * (int32_t)nR;   // kZeroChunks chunks of zero blocks after the row-side chunks
  std::vector<int32_t> Rcol(nR > 0 ? nR : 1), pos(nL > 0 ? nL : 1), Tpos(nT > 0 ? nT : 1), Tsrc(nT > 0 ? nT : 1);
  // row side first: the column side refers to the value positions of later rows
  for (int s = 0; s < ns; ++s) {
    const int lr = (offR[s + 1] - offR[s]) / 32;
    for (int l = 0; l < 32; ++l) {
      const int i = srow[32 * s + l];
      const int len = i >= 0 ? rp[i + 1] - rp[i] : 0;
      for (int k = 0; k < lr; ++k) {
        const int32_t idx = offR[s] + 32 * k + l;
        if (k < len) {
          const int32_t slot = rp[i] + k;
          Rcol[idx] = col[slot];
          pos[slot] = 9 * (idx - l) + l;
        } else {
          Rcol[idx] = i >= 0 ? i : 0;   // padding: a zero block times a valid entry
        }
      }
    }
  }
  for (int s = 0; s < ns; ++s) {
    const int lt = (offT[s + 1] - offT[s]) / 32;
    for (int l = 0; l < 32; ++l) {
      const int i = srow[32 * s + l];
      const int len = i >= 0 ? cp[i + 1] - cp[i] : 0;
      for (int k = 0; k < lt; ++k) {
        const int32_t idx = offT[s] + 32 * k + l;
        if (k < len) {
          Tpos[idx] = pos[cslot[cp[i] + k]];
          Tsrc[idx] = crow[cp[i] + k];
        } else {
          Tpos[idx] = zero + 288 * (s % kZeroChunks) + l;   // padding: a zero chunk
          Tsrc[idx] = i >= 0 ? i : 0;
        }
      }
    }
  }
  std::vector<short2> len((size_t)ns * 32, short2{0, 0});
  for (int i = 0; i < nv; ++i) {
    const int a = rp[i + 1] - rp[i], b = cp[i + 1] - cp[i];
    if (a > 32767 || b > 32767) {
      set_error("df64 pcg: vertex %d has more than 32767 neighbours", i);
      return BAL_ERR_CAPACITY;
    }
    len[slot_of[i]] = short2{(short)a, (short)b};
  }
  BAL_TRY(buf_reserve(S.sell_len, sizeof(short2) * len.size()));
  BAL_CUDA(cudaMemcpy(S.sell_len.p, len.data(), sizeof(short2) * len.size(), cudaMemcpyHostToDevice));
  auto up = [&](Buf& b, const std::vector<int32_t>& v) -> bal_status {
    BAL_TRY(buf_reserve(b, sizeof(int32_t) * v.size()));
    BAL_CUDA(cudaMemcpy(b.p, v.data(), sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice));
    return BAL_OK;
  };
  BAL_TRY(up(S.sell_offR, offR));
  BAL_TRY(up(S.sell_offT, offT));
  BAL_TRY(up(S.sell_Rcol, Rcol));
  BAL_TRY(up(S.sell_Tpos, Tpos));
  BAL_TRY(up(S.sell_Tsrc, Tsrc));
  BAL_TRY(up(S.sell_pos, pos));
  BAL_TRY(up(S.sell_srow, srow));
  BAL_TRY(up(S.sell_slot, slot_of));
  const size_t nRval = 9 * (size_t)(nR + 32 * kZeroChunks), nDval = (size_t)ns * 9 * 32;
  BAL_TRY(buf_reserve(S.dd_R, sizeof(dd) * nRval));
  BAL_TRY(buf_reserve(S.dd_D, sizeof(dd) * nDval));
  BAL_TRY(buf_reserve(S.dd_Dinv, sizeof(dd) * nDval));
  BAL_CUDA(cudaMemset(S.dd_R.p, 0, sizeof(dd) * nRval));   // padding and the zero chunk stay zero
  BAL_CUDA(cudaMemset(S.dd_D.p, 0, sizeof(dd) * nDval));
  BAL_CUDA(cudaMemset(S.dd_Dinv.p, 0, sizeof(dd) * nDval));
  BAL_TRY(buf_reserve(S.dd_vec, sizeof(dd) * 6 * 3 * (size_t)nv));
  S.n_slices = ns;
  S.sell_zero = zero;
  S.sell_built = true;
  S.sell_window = win;
  return BAL_OK;
}

// contact rows of the current C: the vertices touched by C or C^T, each with
// its entries ordered by entry index (a counting sort by vertex, then a rank
// sort inside each vertex's bucket: deterministic, no library sort)
bal_status build_contact_rows(Scene& S, cudaStream_t st) {
  const int nC = (int)S.nnzC, n2 = 2 * nC, nv = S.d.nv;
  S.n_crows = 0;
  if (nC == 0) return BAL_OK;
  BAL_TRY(buf_reserve(S.cr_key, sizeof(uint64_t) * n2));
  for (Buf* b : {&S.cr_bucket, &S.cr_ent, &S.cr_src, &S.cr_rows})
    BAL_TRY(buf_reserve(*b, sizeof(int32_t) * n2));
  BAL_TRY(buf_reserve(S.cr_ptr, sizeof(int32_t) * (n2 + 1)));
  for (Buf* b : {&S.cr_cnt, &S.cr_off, &S.cr_len, &S.cr_rpos})
    BAL_TRY(buf_reserve(*b, sizeof(int32_t) * ((size_t)nv + 1)));
  const int32_t* crow = S.C_row.as<int32_t>();
  const int32_t* ccol = S.C_col.as<int32_t>();
  k_crow_keys<<<grid_for(n2), kThreads, 0, st>>>(crow, ccol, nC, S.cr_key.as<uint64_t>());
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  int32_t* off = S.cr_off.as<int32_t>();
  int32_t* len = S.cr_len.as<int32_t>();
  int32_t* rpos = S.cr_rpos.as<int32_t>();
  BAL_TRY(rows_bucket(S, S.cr_key.as<uint64_t>(), n2, nv, S.cr_cnt.as<int32_t>(), off,
                      S.cr_bucket.as<int32_t>(), S.cr_ent.as<int32_t>(), len, st));
  k_crow_flag<<<grid_for(nv), kThreads, 0, st>>>(len, nv, S.cr_cnt.as<int32_t>());
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  BAL_TRY(scan_i32(S, S.cr_cnt.as<int32_t>(), rpos, nv, st));
  // vertex -> contact row, and room for the contact part of H p per contact row
  BAL_TRY(buf_reserve(S.cr_of, sizeof(int32_t) * (size_t)nv));
  BAL_TRY(buf_reserve(S.cr_q, sizeof(dd) * 3 * (size_t)n2));
  k_crow_rows<<<grid_for(nv), kThreads, 0, st>>>(len, off, rpos, nv, n2, S.cr_rows.as<int32_t>(),
                                                 S.cr_ptr.as<int32_t>(), S.cr_of.as<int32_t>());
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  k_crow_src<<<grid_for(n2), kThreads, 0, st>>>(S.cr_ent.as<int32_t>(), crow, ccol, n2, S.cr_src.as<int32_t>());
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  int32_t n = 0;
  BAL_CUDA(cudaMemcpyAsync(&n, rpos + nv, sizeof(n), cudaMemcpyDeviceToHost, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  S.n_crows = n;
  return BAL_OK;
}

// double-float copies of the assembled H and D^{-1}; contact rows.
// *in_range = false if an entry exceeds the FP32 exponent range.
bal_status refresh_dd(Scene& S, bool* in_range, cudaStream_t st) {
  const int nv = S.d.nv;
  const int64_t nL = S.d.nnzL, nC = S.nnzC;
  if (!S.sell_built || S.sell_window != S.prm.spmv_window) BAL_TRY(build_sell(S, S.prm.spmv_window));
  unsigned int* bad = reinterpret_cast<unsigned int*>(S.scal + 61);
  BAL_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned int), st));
  k_dd_slices<<<grid_for(9 * (int64_t)nv), kThreads, 0, st>>>(nv, S.d.D, S.dd_D.as<dd>(), bad,
                                                               S.sell_slot.as<int32_t>());
  ::bal::note_launch();
  k_dd_slices<<<grid_for(9 * (int64_t)nv), kThreads, 0, st>>>(nv, S.d.Dinv, S.dd_Dinv.as<dd>(), bad, nullptr);
  ::bal::note_launch();
  if (nL) {
    k_dd_scatter<<<grid_for(9 * nL), kThreads, 0, st>>>(nL, S.d.Lval, S.sell_pos.as<int32_t>(),
                                                         S.dd_R.as<dd>(), bad);
    ::bal::note_launch();
  }
  BAL_LAUNCH_CHECK();
  if (nC) {
    BAL_TRY(buf_reserve(S.dd_C, sizeof(dd) * 9 * (size_t)nC));
    k_to_dd<<<grid_for(9 * nC), kThreads, 0, st>>>(9 * nC, S.C_val.as<double>(), S.dd_C.as<dd>(), bad);
    ::bal::note_launch();
    BAL_LAUNCH_CHECK();
  }
  BAL_TRY(build_contact_rows(S, st));
  unsigned int nbad = 0;
  BAL_CUDA(cudaMemcpyAsync(&nbad, bad, sizeof(nbad), cudaMemcpyDeviceToHost, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  *in_range = nbad == 0;
  return BAL_OK;
}

// launch with programmatic stream serialisation (the kernel calls pdl_enter)
template <typename... K, typename... A>
cudaError_t launch_pdl_smem(void (*kernel)(K...), int grid, int block, size_t smem, cudaStream_t st,
                            A&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}
template <typename... K, typename... A>
cudaError_t launch_pdl(void (*kernel)(K...), int grid, int block, cudaStream_t st, A&&... args) {
  return launch_pdl_smem(kernel, grid, block, 0, st, std::forward<A>(args)...);
}

DDSys dd_sys(Scene& S) {
  DDSys A;
  A.D = S.dd_D.as<dd>();
  A.Dinv = S.dd_Dinv.as<dd>();
  A.offR = S.sell_offR.as<int32_t>();
  A.Rcol = S.sell_Rcol.as<int32_t>();
  A.R = S.dd_R.as<dd>();
  A.offT = S.sell_offT.as<int32_t>();
  A.Tpos = S.sell_Tpos.as<int32_t>();
  A.Tsrc = S.sell_Tsrc.as<int32_t>();
  A.len = S.sell_len.as<short2>();
  A.srow = S.sell_srow.as<int32_t>();
  A.zero = S.sell_zero;
  A.nv = S.d.nv;
  A.ns = S.n_slices;
  return A;
}

DDContact dd_contact(Scene& S) {
  DDContact C;
  C.rows = S.cr_rows.as<int32_t>();
  C.ptr = S.cr_ptr.as<int32_t>();
  C.ent = S.cr_ent.as<int32_t>();
  C.src = S.cr_src.as<int32_t>();
  C.C = S.dd_C.as<dd>();
  C.n = S.n_crows;
  return C;
}

}  // namespace

bal_status pcg_df64(Scene& S, const double* b, double* x, double tol, int max_it,
                    bal_solve_info* info, cudaStream_t st) {
  bool in_range = true;
  if (!S.dd_valid || S.sell_window != S.prm.spmv_window) {
    BAL_TRY(refresh_dd(S, &in_range, st));
    S.dd_valid = in_range;
  }
  if (!in_range) {   // an entry outside the FP32 exponent range: the FP64 solver takes it
    const int32_t keep = S.prm.precision, keep_pc = S.prm.precond;
    S.prm.precision = BAL_PREC_FP64;
    S.prm.precond = BAL_PRECOND_BJ;   // a requested warm start has already run
    const bal_status s = pcg_solve(S, b, x, tol, max_it, info, st);
    S.prm.precision = keep;
    S.prm.precond = keep_pc;
    if (info) info->precision_used = BAL_PREC_FP64;
    return s;
  }
  const int nv = S.d.nv;
  const int64_t n3 = 3 * (int64_t)nv;
  const DDSys A = dd_sys(S);
  const DDContact Cr = dd_contact(S);
  dd* V = S.dd_vec.as<dd>();
  dd *ex = V, *er = V + n3, *ez = V + 2 * n3, *ep = V + 3 * n3, *eq = V + 4 * n3;
  const int W = S.sell_window;   // 0: row-gather kernel; > 0: windowed kernel
  const int gs = W > 0 ? (nv + W - 1) / W : std::min((S.n_slices + kDdWarps - 1) / kDdWarps, kMaxPartials / 2);
  const size_t smem_w = W > 0 ? (size_t)W * 3 * (sizeof(double) + sizeof(dd)) : 0;
  if (W > 0) {
    if (gs > kMaxPartials / 2) {
      set_error("df64 pcg: %d windows of %d rows exceed the %d partial sums", gs, W, kMaxPartials / 2);
      return BAL_ERR_CAPACITY;
    }
    BAL_CUDA(cudaFuncSetAttribute(k_dd_spmv_win, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_w));
  }
  const int gv = std::min((nv + kDdThreads - 1) / kDdThreads, kMaxPartials / 2);   // one vertex per thread
  // the update kernel takes two vertices per thread when that still leaves
  // at least 4 CTAs per SM
  const int gu = (gv + 1) / 2 >= 4 * kNumSM ? (gv + 1) / 2 : gv;
  // contact CTAs appended to the SpMV grid (none without contact)
  const int gc = Cr.n > 0 ? std::max(1, std::min((int)(((int64_t)Cr.n * kContactLanes + kDdThreads - 1) /
                                                       kDdThreads), kMaxPartials / 2))
                          : 0;
  const int32_t* crow_of = Cr.n > 0 ? S.cr_of.as<int32_t>() : nullptr;
  dd* eqc = S.cr_q.as<dd>();
  double rn, bn;
  BAL_TRY(residual_fp64(S, b, x, S.pcg_r, &rn, &bn, st));
  const double r0 = rn;
  int total = 0, passes = 0, stagnated = 0;
  bool converged = rn <= tol * r0 || rn == 0.0;
  while (!converged && passes <= S.prm.mixed_max_refine && total < max_it) {
    // solve H e = r / ||r|| to tol * r0 / ||r||, then x += ||r|| e
    PcgScalars init{};
    init.max_it = max_it - total;
    init.window = S.prm.pcg_stall_window > 0 ? S.prm.pcg_stall_window : (1 << 30);
    init.stall_rel = S.prm.pcg_stall_forcing > 0 ? S.prm.pcg_stall_forcing : INFINITY;
    BAL_CUDA(cudaMemcpyAsync(S.pcg, &init, sizeof(init), cudaMemcpyHostToDevice, st));
    k_dd_init<kDdThreads><<<gv, kDdThreads, 0, st>>>(A, S.pcg_r, 1.0 / rn, ex, er, ez, S.pcg,
                                                            S.partials, tol * r0 / rn);
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
      if (h.done || launched >= init.max_it) break;
      const int n = std::min(chunk, init.max_it - launched);
      for (int k = 0; k < n; ++k) {
        BAL_CUDA(launch_pdl(k_dd_dir<kDdThreads>, gv, kDdThreads, st, nv, (const dd*)ez, ep,
                            (const PcgScalars*)S.pcg));
        ::bal::note_launch();
        // one SpMV per chunk is timed: an event between two launches ends
        // their programmatic overlap
        if (k == 0) kt_before(S, 0, st);
        if (W > 0)
          BAL_CUDA(launch_pdl_smem(k_dd_spmv_win, gs + gc, kDdThreads, smem_w, st, A, Cr, gs, W, (const dd*)ep,
                                   eq, eqc, S.pcg, S.partials));
        else
          BAL_CUDA(launch_pdl(k_dd_spmv, gs + gc, kDdThreads, st, A, Cr, gs, (const dd*)ep, eq, eqc, S.pcg,
                              S.partials));
        if (k == 0) {
          kt_after(S, 0, st);
          ++timed;
        }
        ::bal::note_launch();
        BAL_CUDA(launch_pdl(k_dd_update<kDdThreads>, gu, kDdThreads, st, A, ex, (const dd*)ep,
                            (const dd*)eq, crow_of, (const dd*)eqc, er, ez, S.pcg, S.partials));
        ::bal::note_launch();
      }
      BAL_LAUNCH_CHECK();
      launched += n;
    }
    if (h.done == 2 || h.done == 3) {
      set_error("df64 pcg: %s at iteration %d", h.done == 2 ? "non-finite residual" : "p^T H p <= 0",
                total + h.it);
      return BAL_ERR_NAN;
    }
    total += h.it;
    passes += 1;
    stagnated = h.stagnated;
    k_dd_accumulate<<<grid_for(n3), kThreads, 0, st>>>(n3, rn, ex, x);
    ::bal::note_launch();
    BAL_LAUNCH_CHECK();
    const double prev = rn;
    BAL_TRY(residual_fp64(S, b, x, S.pcg_r, &rn, &bn, st));
    if (!std::isfinite(rn)) {
      set_error("df64 pcg: non-finite FP64 residual after pass %d", passes);
      return BAL_ERR_NAN;
    }
    converged = rn <= tol * r0;
    // a pass that ended by stagnation or the cap, or made no progress, ends the solve
    if (!h.converged || !(rn < 0.99 * prev) || h.it == 0) break;
  }
  if (info) {
    info->iters = total;
    info->rel_residual = bn > 0 ? rn / bn : rn;
    info->rel_residual_r0 = r0 > 0 ? rn / r0 : rn;
    info->stagnated = converged ? 0 : stagnated;
    info->converged = converged ? 1 : 0;
    info->refine_passes = passes > 0 ? passes - 1 : 0;
    info->warm_iters = 0;
    info->n_groups = 0;
    info->negative_curvature = 0;
    info->precision_used = BAL_PREC_DF64;
  }
  return BAL_OK;
}

}  // namespace bal
