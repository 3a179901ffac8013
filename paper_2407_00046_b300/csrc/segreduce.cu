// Merge of the duplicate contact blocks of the BSR assembly (Sec. 5.1, App. C:
// every contact stencil emits its 6 off-diagonal lower 3x3 blocks; blocks that
// land on the same (row, col) are summed into the C part of the symmetric
// storage). Hand-written, no library sort:
//
//   1. counting sort by row: per-row counts (atomics), exclusive scan, scatter
//      of the record indices into per-row buckets;
//   2. inside each row, one warp orders the bucket by (col, emission index) --
//      a rank sort, with the keys held in registers and exchanged by shuffles
//      when the row has at most 32 records -- and counts the distinct columns;
//   3. exclusive scan of those counts gives every merged block its slot;
//   4. one warp per row sums each run of equal columns with a warp-segmented
//      inclusive scan over the 9 block values (carried across 32-record
//      chunks) and the last lane of each run writes the merged block.
//
// The order of every sum is fixed by (col, emission index), so the merged
// values are bit-reproducible for a given emission. Output: C sorted by
// (row, col), as the rest of the library expects.
#include "scene.cuh"

namespace bal {

namespace {

constexpr int kScanNT = 1024;        // scan CTA size
constexpr int kScanItems = 4;        // elements per thread
constexpr int kScanTile = kScanNT * kScanItems;

// exclusive prefix of v over the CTA; *total gets the CTA sum
__device__ inline int32_t cta_exclusive_scan(int32_t v, int32_t* total) {
  __shared__ int32_t wsum[kScanNT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int32_t s = wsum[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= d) s += y;
    }
    wsum[lane] = s;   // inclusive prefix of the warp sums
  }
  __syncthreads();
  const int32_t excl = x - v + (w > 0 ? wsum[w - 1] : 0);
  *total = wsum[kScanNT / 32 - 1];
  __syncthreads();   // wsum is reused by the next call
  return excl;
}

// phase 1: tile-local exclusive scan of in[0, n) into out, tile sums into aux
__global__ void __launch_bounds__(kScanNT) k_scan_tiles(const int32_t* __restrict__ in, int64_t n,
                                                        int32_t* __restrict__ out, int32_t* __restrict__ aux) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems], s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    s += v[k];
  }
  int32_t tot;
  int32_t run = cta_exclusive_scan(s, &tot);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) aux[blockIdx.x] = tot;
}

// phase 2: exclusive scan of the tile sums in place (one CTA, chunks with a
// carry); aux[ntiles] = grand total
__global__ void __launch_bounds__(kScanNT) k_scan_aux(int32_t* aux, int ntiles) {
  __shared__ int32_t carry_sh;
  if (threadIdx.x == 0) carry_sh = 0;
  __syncthreads();
  for (int c = 0; c < ntiles; c += kScanNT) {
    const int i = c + threadIdx.x;
    const int32_t v = i < ntiles ? aux[i] : 0;
    int32_t tot;
    const int32_t ex = cta_exclusive_scan(v, &tot);
    const int32_t carry = carry_sh;
    if (i < ntiles) aux[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry_sh = carry + tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) aux[ntiles] = carry_sh;
}

// phase 3: add each tile's offset; out[n] = total
__global__ void __launch_bounds__(kScanNT) k_scan_add(int32_t* __restrict__ out, int64_t n,
                                                      const int32_t* __restrict__ aux, int ntiles) {
  const int32_t off = aux[blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int k = threadIdx.x; k < kScanTile; k += kScanNT)
    if (base + k < n) out[base + k] += off;
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = aux[ntiles];
}

// ---- duplicate-block merge ------------------------------------------------------
__device__ inline int32_t key_row(uint64_t k) { return (int32_t)(k >> 32); }
__device__ inline int32_t key_col(uint64_t k) { return (int32_t)(k & 0xffffffffu); }

__global__ void k_cm_count(const uint64_t* __restrict__ keys, int64_t n, int32_t* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    if (k != ~0ull) atomicAdd(cnt + key_row(k), 1);
  }
}

__global__ void k_cm_scatter(const uint64_t* __restrict__ keys, int64_t n, const int32_t* __restrict__ off,
                             int32_t* __restrict__ fill, int32_t* __restrict__ bucket) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    if (k == ~0ull) continue;
    const int32_t r = key_row(k);
    bucket[off[r] + atomicAdd(fill + r, 1)] = (int32_t)i;
  }
}

// sort key of a record inside its row: column, then emission index
__device__ inline uint64_t rank_key(const uint64_t* __restrict__ keys, int32_t idx) {
  return ((uint64_t)(uint32_t)key_col(keys[idx]) << 32) | (uint32_t)idx;
}

// one warp per row: order the bucket by (col, emission index) into `sorted`
// and count the distinct columns into ucnt
__global__ void k_cm_order(const uint64_t* __restrict__ keys, const int32_t* __restrict__ off, int nv,
                           const int32_t* __restrict__ bucket, int32_t* __restrict__ sorted,
                           int32_t* __restrict__ ucnt) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nv; r += warps) {
    const int32_t b = off[r], L = off[r + 1] - b;
    if (L == 0) {
      if (lane == 0) ucnt[r] = 0;
      continue;
    }
    int32_t heads = 0;
    if (L <= 32) {
      const int32_t idx = lane < L ? bucket[b + lane] : 0;
      const uint64_t mk = lane < L ? rank_key(keys, idx) : ~0ull;
      int32_t rank = 0;
      bool head = true;
      for (int j = 0; j < L; ++j) {
        const uint64_t kj = __shfl_sync(0xffffffffu, mk, j);
        rank += kj < mk;
        head = head && !((kj >> 32) == (mk >> 32) && kj < mk);
      }
      if (lane < L) {
        sorted[b + rank] = idx;
        heads = head ? 1 : 0;
      }
    } else {
      for (int e = lane; e < L; e += 32) {
        const int32_t idx = bucket[b + e];
        const uint64_t mk = rank_key(keys, idx);
        int32_t rank = 0;
        bool head = true;
        for (int j = 0; j < L; ++j) {
          const uint64_t kj = rank_key(keys, bucket[b + j]);
          rank += kj < mk;
          head = head && !((kj >> 32) == (mk >> 32) && kj < mk);
        }
        sorted[b + rank] = idx;
        heads += head ? 1 : 0;
      }
    }
    heads = warp_sum(heads);
    if (lane == 0) ucnt[r] = heads;
  }
}

// one warp per row: warp-segmented sums of the runs of equal columns
__global__ void k_cm_reduce(const uint64_t* __restrict__ keys, const double* __restrict__ vals,
                            const int32_t* __restrict__ off, const int32_t* __restrict__ uoff, int nv,
                            const int32_t* __restrict__ sorted, int32_t* __restrict__ crow,
                            int32_t* __restrict__ ccol, double* __restrict__ cval) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nv; r += warps) {
    const int32_t b = off[r], L = off[r + 1] - b;
    if (L == 0) continue;
    int32_t out = uoff[r] - 1;        // slot of the current run (advanced at each head)
    int32_t carry_col = -1;           // column of the run open at the end of the last chunk
    double carry[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) carry[c] = 0.0;
    for (int e0 = 0; e0 < L; e0 += 32) {
      const int e = e0 + lane;
      const bool live = e < L;
      const int32_t idx = live ? sorted[b + e] : 0;
      const int32_t col = live ? key_col(keys[idx]) : -2;
      double v[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) v[c] = live ? vals[9 * (int64_t)idx + c] : 0.0;
      const int32_t prev = __shfl_up_sync(0xffffffffu, col, 1);
      const bool head = live && (lane == 0 ? col != carry_col : col != prev);
      if (lane == 0 && !head) {       // continue the run of the previous chunk
#pragma unroll
        for (int c = 0; c < 9; ++c) v[c] += carry[c];
      }
      // segmented inclusive scan: f = "a head lies in my window"
      bool f = head;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const bool fu = __shfl_up_sync(0xffffffffu, f, d);
        double u[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) u[c] = __shfl_up_sync(0xffffffffu, v[c], d);
        if (lane >= d && !f) {
#pragma unroll
          for (int c = 0; c < 9; ++c) v[c] += u[c];
        }
        if (lane >= d) f = f || fu;
      }
      // slot of my run: heads so far in this row
      const unsigned hm = __ballot_sync(0xffffffffu, head);
      const int32_t slot = out + __popc(hm & ((2u << lane) - 1u));
      const int32_t next = __shfl_down_sync(0xffffffffu, col, 1);
      const bool last_in_chunk = lane == 31 || !(e + 1 < L);
      if (live && !last_in_chunk && next != col) {
        crow[slot] = r;
        ccol[slot] = col;
#pragma unroll
        for (int c = 0; c < 9; ++c) cval[9 * (int64_t)slot + c] = v[c];
      }
      // the run open at the end of the chunk: written here when it ends with
      // the chunk (end of the row, or the next chunk starts another column),
      // otherwise carried into the next chunk
      const int tail = min(31, L - 1 - e0);
      const int32_t tcol = __shfl_sync(0xffffffffu, col, tail);
      const int32_t tslot = __shfl_sync(0xffffffffu, slot, tail);
#pragma unroll
      for (int c = 0; c < 9; ++c) carry[c] = __shfl_sync(0xffffffffu, v[c], tail);
      const bool more = e0 + 32 < L;
      const int32_t ncol = more ? key_col(keys[sorted[b + e0 + 32]]) : -3;
      if (!more || ncol != tcol) {
        if (lane == 0) {
          crow[tslot] = r;
          ccol[tslot] = tcol;
#pragma unroll
          for (int c = 0; c < 9; ++c) cval[9 * (int64_t)tslot + c] = carry[c];
        }
        carry_col = -1;
      } else {
        carry_col = tcol;
      }
      out += __popc(hm);
    }
  }
}

}  // namespace

// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total (int32).
bal_status scan_i32(Scene& S, const int32_t* in, int32_t* out, int64_t n, cudaStream_t st) {
  const int ntiles = (int)((n + kScanTile - 1) / kScanTile);
  if (ntiles == 0) {
    BAL_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), st));
    return BAL_OK;
  }
  BAL_TRY(buf_reserve(S.scan_aux, sizeof(int32_t) * (ntiles + 1)));
  int32_t* aux = S.scan_aux.as<int32_t>();
  k_scan_tiles<<<ntiles, kScanNT, 0, st>>>(in, n, out, aux);
  k_scan_aux<<<1, kScanNT, 0, st>>>(aux, ntiles);
  k_scan_add<<<ntiles, kScanNT, 0, st>>>(out, n, aux, ntiles);
  ::bal::note_launch(3);
  BAL_LAUNCH_CHECK();
  return BAL_OK;
}

// Counting sort of n records (keys[i] = row << 32 | col, ~0 = dropped) into
// per-row buckets, each ordered by (col, record index): off[0..nv] are the
// bucket offsets, sorted[off[r] .. off[r+1]) the record indices of row r and
// ucnt[r] its number of distinct columns. cnt ([nv + 1]) and bucket ([n]) are
// scratch. No host synchronisation.
bal_status rows_bucket(Scene& S, const uint64_t* keys, int64_t n, int nv, int32_t* cnt, int32_t* off,
                       int32_t* bucket, int32_t* sorted, int32_t* ucnt, cudaStream_t st) {
  const size_t nrow = (size_t)nv + 1;
  BAL_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * nrow, st));
  k_cm_count<<<grid_for(n), kThreads, 0, st>>>(keys, n, cnt);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  BAL_TRY(scan_i32(S, cnt, off, nv, st));
  BAL_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * nrow, st));   // reused as the fill counters
  k_cm_scatter<<<grid_for(n), kThreads, 0, st>>>(keys, n, off, cnt, bucket);
  ::bal::note_launch();
  const int row_blocks = grid_for((int64_t)nv * 32, kThreads, kNumSM * 16);
  k_cm_order<<<row_blocks, kThreads, 0, st>>>(keys, off, nv, bucket, sorted, ucnt);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  return BAL_OK;
}

// Merge the n_emit emitted contact blocks (S.emit_keys: row << 32 | col, ~0 =
// dropped; S.emit_vals: [n_emit][9]) into C (S.C_row, S.C_col, S.C_val, S.nnzC),
// sorted by (row, col).
bal_status contact_blocks_reduce(Scene& S, int64_t n_emit, cudaStream_t st) {
  S.nnzC = 0;
  if (n_emit <= 0) return BAL_OK;
  const int nv = S.d.nv;
  const size_t nrow = (size_t)nv + 1;
  for (Buf* b : {&S.cm_cnt, &S.cm_off, &S.cm_ucnt, &S.cm_uoff})
    BAL_TRY(buf_reserve(*b, sizeof(int32_t) * nrow));
  BAL_TRY(buf_reserve(S.cm_bucket, sizeof(int32_t) * n_emit));
  BAL_TRY(buf_reserve(S.cm_sorted, sizeof(int32_t) * n_emit));
  const uint64_t* keys = S.emit_keys.as<uint64_t>();
  int32_t* off = S.cm_off.as<int32_t>();
  BAL_TRY(rows_bucket(S, keys, n_emit, nv, S.cm_cnt.as<int32_t>(), off, S.cm_bucket.as<int32_t>(),
                      S.cm_sorted.as<int32_t>(), S.cm_ucnt.as<int32_t>(), st));
  const int row_blocks = grid_for((int64_t)nv * 32, kThreads, kNumSM * 16);
  int32_t* uoff = S.cm_uoff.as<int32_t>();
  BAL_TRY(scan_i32(S, S.cm_ucnt.as<int32_t>(), uoff, nv, st));
  int32_t nC = 0;
  BAL_CUDA(cudaMemcpyAsync(&nC, uoff + nv, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  BAL_TRY(buf_reserve(S.C_row, sizeof(int32_t) * (nC + 1)));
  BAL_TRY(buf_reserve(S.C_col, sizeof(int32_t) * (nC + 1)));
  BAL_TRY(buf_reserve(S.C_val, sizeof(double) * 9 * (nC + 1)));
  if (nC > 0) {
    k_cm_reduce<<<row_blocks, kThreads, 0, st>>>(keys, S.emit_vals.as<double>(), off, uoff, nv,
                                                 S.cm_sorted.as<int32_t>(), S.C_row.as<int32_t>(),
                                                 S.C_col.as<int32_t>(), S.C_val.as<double>());
    ::bal::note_launch();
    BAL_LAUNCH_CHECK();
  }
  S.nnzC = nC;
  return BAL_OK;
}

}  // namespace bal
