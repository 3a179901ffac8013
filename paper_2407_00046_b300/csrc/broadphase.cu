// Broad phase: uniform-grid hash over the boundary primitives. Produces every
// point-triangle and edge-edge pair (not sharing a vertex) whose primitives'
// axis-aligned boxes come within r of each other -- a superset of the pairs
// with distance below r -- each pair exactly once, sorted by pair key.
//
// Every primitive has an inflation radius r_P (uniform, or from its nodes'
// displacements, see Grid). Triangles (for PT) and edges (for EE) are inserted,
// with their boxes inflated by their own r, into every cell the box overlaps.
// A query primitive (surface vertex, or edge e) scans the cells overlapped by
// its own inflated box and keeps a pair only if the two inflated boxes overlap
// and the cell holds the lower corner of their intersection, so a pair seen in
// several cells is reported once. Large radii only enlarge their own
// primitive's cell range, never the grid.
// (The paper's broad phase is an LBVH, Sec. 5.3; the grid is this build's.)
#include <cub/cub.cuh>
#include <cstring>
#include <vector>

#include "scene.cuh"

namespace bal {

namespace {

// cell key: 16 bits per axis (bits 16..63) + 16 bits of body id (motion passes)
constexpr int kOff = 1 << 15;
constexpr uint32_t kBodySat = 0xffffu;   // body ids >= this share one id (no skipping)
constexpr int64_t kMaxCellsPerPrim = 1 << 20;

// Per-vertex inflation radius r_v; a primitive's radius is the max over its
// nodes. Pairs (P, Q) are kept when their boxes inflated by r_P and r_Q overlap.
//   uniform (mode 0): r_v = r/2, every pair, so boxes within r are kept;
//   motion (mode 1 / 2): r_v = (|p_v - pbar_B| [+ |pbar_B|]) / eta + dhat/2 with
//     pbar_B the mean displacement of v's body; mode 1 keeps same-body pairs
//     only (no |pbar_B| term), mode 2 different-body pairs only.
struct Grid {
  double inv_c;
  double half_r;     // uniform: r/2
  double rmax;       // typical r_v of this pass (sets the cell size only)
  int mode;
  const double* dir;
  const double* bmean;   // [nbody][3]
  const double* bmot;    // [nbody] half the largest mean relative motion to an interacting body
  const int32_t* body;   // [nv]
  double eta, base;
};

__device__ inline double vert_r(const Grid& G, int v) {
  if (G.mode == 0) return G.half_r;
  const int b = G.body[v];
  const d3 pb = d3{G.bmean[3 * b], G.bmean[3 * b + 1], G.bmean[3 * b + 2]};
  const d3 w = ld3(G.dir, v) - pb;
  double r = sqrt(dot(w, w));
  if (G.mode == 2) r += G.bmot[b];
  return r / G.eta + G.base;
}
__device__ inline uint32_t body_bits(const Grid& G, int v) {
  if (G.mode == 0) return 0u;
  const uint32_t b = (uint32_t)G.body[v];
  return b < kBodySat ? b : kBodySat;
}
__device__ inline bool body_ok(const Grid& G, int va, int vb) {
  if (G.mode == 0) return true;
  return G.mode == 1 ? G.body[va] == G.body[vb] : G.body[va] != G.body[vb];
}

__device__ inline int cell_of(double v, double inv_c) {
  double f = floor(v * inv_c);
  f = fmin(fmax(f, -(double)(kOff - 1)), (double)(kOff - 1));
  return (int)f;
}
__device__ inline uint64_t cell_key(int ix, int iy, int iz) {
  return ((uint64_t)(ix + kOff) << 48) | ((uint64_t)(iy + kOff) << 32) | ((uint64_t)(iz + kOff) << 16);
}

struct Box {
  d3 lo, hi;
};
__device__ inline Box prim_box(const double* x, const int* v, int nv) {
  Box b;
  b.lo = ld3(x, v[0]);
  b.hi = b.lo;
  for (int k = 1; k < nv; ++k) {
    const d3 p = ld3(x, v[k]);
    b.lo = d3{fmin(b.lo.x, p.x), fmin(b.lo.y, p.y), fmin(b.lo.z, p.z)};
    b.hi = d3{fmax(b.hi.x, p.x), fmax(b.hi.y, p.y), fmax(b.hi.z, p.z)};
  }
  return b;
}
__device__ inline Box inflate(Box b, double r) {
  return Box{d3{b.lo.x - r, b.lo.y - r, b.lo.z - r}, d3{b.hi.x + r, b.hi.y + r, b.hi.z + r}};
}
__device__ inline bool overlap(const Box& a, const Box& b) {
  return a.lo.x <= b.hi.x && b.lo.x <= a.hi.x && a.lo.y <= b.hi.y && b.lo.y <= a.hi.y &&
         a.lo.z <= b.hi.z && b.lo.z <= a.hi.z;
}

__device__ inline void prim_verts(const Dev& S, int kind, int id, int v[3], int& nv) {
  if (kind == 0) {
    v[0] = S.tris[3 * (int64_t)id];
    v[1] = S.tris[3 * (int64_t)id + 1];
    v[2] = S.tris[3 * (int64_t)id + 2];
    nv = 3;
  } else {
    v[0] = S.edges[2 * (int64_t)id];
    v[1] = S.edges[2 * (int64_t)id + 1];
    nv = 2;
  }
}

__device__ inline double prim_r(const Grid& G, const int* v, int nv) {
  double r = vert_r(G, v[0]);
  for (int k = 1; k < nv; ++k) r = fmax(r, vert_r(G, v[k]));
  return r;
}

// number of cells of each inflated primitive box (kind 0 = triangles, 1 = edges)
__global__ void k_count_cells(Dev S, const double* __restrict__ x, int kind, int n, Grid G,
                              int64_t* __restrict__ count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int v[3], nv;
    prim_verts(S, kind, i, v, nv);
    const Box b = inflate(prim_box(x, v, nv), prim_r(G, v, nv));
    const int64_t c = (int64_t)(cell_of(b.hi.x, G.inv_c) - cell_of(b.lo.x, G.inv_c) + 1) *
                      (cell_of(b.hi.y, G.inv_c) - cell_of(b.lo.y, G.inv_c) + 1) *
                      (cell_of(b.hi.z, G.inv_c) - cell_of(b.lo.z, G.inv_c) + 1);
    count[i] = c > kMaxCellsPerPrim ? kMaxCellsPerPrim : c;
  }
}

__global__ void k_fill_cells(Dev S, const double* __restrict__ x, int kind, int n, Grid G,
                             const int64_t* __restrict__ offs, uint64_t* __restrict__ cells,
                             int32_t* __restrict__ ids) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int v[3], nv;
    prim_verts(S, kind, i, v, nv);
    const Box b = inflate(prim_box(x, v, nv), prim_r(G, v, nv));
    const int x0 = cell_of(b.lo.x, G.inv_c), x1 = cell_of(b.hi.x, G.inv_c);
    const int y0 = cell_of(b.lo.y, G.inv_c), y1 = cell_of(b.hi.y, G.inv_c);
    const int z0 = cell_of(b.lo.z, G.inv_c), z1 = cell_of(b.hi.z, G.inv_c);
    int64_t o = offs[i];
    const int64_t end = offs[i + 1];
    for (int ix = x0; ix <= x1; ++ix)
      for (int iy = y0; iy <= y1; ++iy)
        for (int iz = z0; iz <= z1; ++iz) {
          if (o >= end) return;
          cells[o] = cell_key(ix, iy, iz) | body_bits(G, v[0]);
          ids[o] = i;
          ++o;
        }
  }
}

__device__ inline int64_t lower_bound(const uint64_t* a, int64_t n, uint64_t k) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] < k) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// entries of one cell a query of body bits qb has to look at: [a0,a1) and [b0,b1)
__device__ inline void cell_ranges(const Grid& G, const uint64_t* cells, int64_t n, uint64_t base,
                                   uint32_t qb, int64_t& a0, int64_t& a1, int64_t& b0, int64_t& b1) {
  const int64_t lo = lower_bound(cells, n, base), hi = lower_bound(cells, n, base + 0x10000ull);
  if (G.mode == 0 || qb == kBodySat) {
    a0 = lo; a1 = hi; b0 = b1 = hi;
    return;
  }
  const int64_t ml = lower_bound(cells, n, base | qb), mh = lower_bound(cells, n, (base | qb) + 1);
  if (G.mode == 1) {        // same body only
    a0 = ml; a1 = mh; b0 = b1 = mh;
  } else {                  // other bodies only
    a0 = lo; a1 = ml; b0 = mh; b1 = hi;
  }
}

__device__ inline void emit(uint64_t* out, unsigned long long* counter, int64_t cap, uint64_t key) {
  const unsigned long long idx = atomicAdd(counter, 1ull);
  if ((int64_t)idx < cap) out[idx] = key;
}

__device__ inline bool canonical(const Box& a, const Box& b, int ix, int iy, int iz, double inv_c) {
  const d3 lo = d3{fmax(a.lo.x, b.lo.x), fmax(a.lo.y, b.lo.y), fmax(a.lo.z, b.lo.z)};
  return cell_of(lo.x, inv_c) == ix && cell_of(lo.y, inv_c) == iy && cell_of(lo.z, inv_c) == iz;
}

__global__ void k_pt_query(Dev S, const double* __restrict__ x, Grid G,
                           const uint64_t* __restrict__ cells, const int32_t* __restrict__ ids,
                           int64_t ncell, uint64_t* out, unsigned long long* counter, int64_t cap) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.nsv; i += gridDim.x * blockDim.x) {
    const int v = S.surf[i];
    const d3 p = ld3(x, v);
    const double rv = vert_r(G, v);
    const Box bp = Box{d3{p.x - rv, p.y - rv, p.z - rv}, d3{p.x + rv, p.y + rv, p.z + rv}};
    const int x0 = cell_of(bp.lo.x, G.inv_c), x1 = cell_of(bp.hi.x, G.inv_c);
    const int y0 = cell_of(bp.lo.y, G.inv_c), y1 = cell_of(bp.hi.y, G.inv_c);
    const int z0 = cell_of(bp.lo.z, G.inv_c), z1 = cell_of(bp.hi.z, G.inv_c);
    for (int ix = x0; ix <= x1; ++ix)
      for (int iy = y0; iy <= y1; ++iy)
        for (int iz = z0; iz <= z1; ++iz) {
          int64_t r0, r1, r2, r3;
          cell_ranges(G, cells, ncell, cell_key(ix, iy, iz), body_bits(G, v), r0, r1, r2, r3);
          for (int64_t kk = r0; kk < r3; ++kk) {
            if (kk == r1) kk = r2;
            if (kk >= r3) break;
            const int t = ids[kk];
            int tv[3], nv;
            prim_verts(S, 0, t, tv, nv);
            if (tv[0] == v || tv[1] == v || tv[2] == v) continue;
            if (!body_ok(G, v, tv[0])) continue;
            const Box bt = inflate(prim_box(x, tv, 3), prim_r(G, tv, 3));
            if (!overlap(bp, bt) || !canonical(bp, bt, ix, iy, iz, G.inv_c)) continue;
            emit(out, counter, cap, pair_key(0, (uint32_t)v, (uint32_t)t));
          }
        }
  }
}

__global__ void k_ee_query(Dev S, const double* __restrict__ x, Grid G,
                           const uint64_t* __restrict__ cells, const int32_t* __restrict__ ids,
                           int64_t ncell, uint64_t* out, unsigned long long* counter, int64_t cap) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < S.ne; e += gridDim.x * blockDim.x) {
    int ev[3], nv;
    prim_verts(S, 1, e, ev, nv);
    const Box be = inflate(prim_box(x, ev, 2), prim_r(G, ev, 2));
    const int x0 = cell_of(be.lo.x, G.inv_c), x1 = cell_of(be.hi.x, G.inv_c);
    const int y0 = cell_of(be.lo.y, G.inv_c), y1 = cell_of(be.hi.y, G.inv_c);
    const int z0 = cell_of(be.lo.z, G.inv_c), z1 = cell_of(be.hi.z, G.inv_c);
    for (int ix = x0; ix <= x1; ++ix)
      for (int iy = y0; iy <= y1; ++iy)
        for (int iz = z0; iz <= z1; ++iz) {
          int64_t r0, r1, r2, r3;
          cell_ranges(G, cells, ncell, cell_key(ix, iy, iz), body_bits(G, ev[0]), r0, r1, r2, r3);
          for (int64_t kk = r0; kk < r3; ++kk) {
            if (kk == r1) kk = r2;
            if (kk >= r3) break;
            const int f = ids[kk];
            if (f <= e) continue;
            int fv[3];
            prim_verts(S, 1, f, fv, nv);
            if (fv[0] == ev[0] || fv[0] == ev[1] || fv[1] == ev[0] || fv[1] == ev[1]) continue;
            if (!body_ok(G, ev[0], fv[0])) continue;
            const Box bf = inflate(prim_box(x, fv, 2), prim_r(G, fv, 2));
            if (!overlap(be, bf) || !canonical(be, bf, ix, iy, iz, G.inv_c)) continue;
            emit(out, counter, cap, pair_key(1, (uint32_t)e, (uint32_t)f));
          }
        }
  }
}

// Builds the sorted (cell, primitive) list of one primitive kind.
bal_status build_cells(Scene& S, const double* x, int kind, int n, Grid G, int64_t* ncell,
                       uint64_t** cells_out, int32_t** ids_out, cudaStream_t st) {
  *ncell = 0;
  if (n == 0) return BAL_OK;
  BAL_TRY(buf_reserve(S.bp_count, sizeof(int64_t) * (n + 1)));
  BAL_TRY(buf_reserve(S.bp_offs, sizeof(int64_t) * (n + 1)));
  int64_t* cnt = S.bp_count.as<int64_t>();
  int64_t* offs = S.bp_offs.as<int64_t>();
  k_count_cells<<<grid_for(n), kThreads, 0, st>>>(S.d, x, kind, n, G, cnt);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  BAL_CUDA(cudaMemsetAsync(cnt + n, 0, sizeof(int64_t), st));
  size_t tmp = 0;
  BAL_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp, cnt, offs, n + 1, st));
  BAL_TRY(buf_reserve(S.cub_tmp, tmp));
  BAL_CUDA(cub::DeviceScan::ExclusiveSum(S.cub_tmp.p, tmp, cnt, offs, n + 1, st));
  int64_t total = 0;
  BAL_CUDA(cudaMemcpyAsync(&total, offs + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  if (total > (int64_t)1 << 31) {
    set_error("broad phase: %lld (cell, primitive) entries; query radius too large", (long long)total);
    return BAL_ERR_CAPACITY;
  }
  BAL_TRY(buf_reserve(S.bp_cells, sizeof(uint64_t) * total));
  BAL_TRY(buf_reserve(S.bp_cells_alt, sizeof(uint64_t) * total));
  BAL_TRY(buf_reserve(S.bp_ids, sizeof(int32_t) * total));
  BAL_TRY(buf_reserve(S.bp_ids_alt, sizeof(int32_t) * total));
  k_fill_cells<<<grid_for(n), kThreads, 0, st>>>(S.d, x, kind, n, G, offs,
                                                 S.bp_cells.as<uint64_t>(), S.bp_ids.as<int32_t>());
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  cub::DoubleBuffer<uint64_t> dk(S.bp_cells.as<uint64_t>(), S.bp_cells_alt.as<uint64_t>());
  cub::DoubleBuffer<int32_t> dv(S.bp_ids.as<int32_t>(), S.bp_ids_alt.as<int32_t>());
  tmp = 0;
  BAL_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp, dk, dv, (int64_t)total, 0, 64, st));
  BAL_TRY(buf_reserve(S.cub_tmp, tmp));
  BAL_CUDA(cub::DeviceRadixSort::SortPairs(S.cub_tmp.p, tmp, dk, dv, (int64_t)total, 0, 64, st));
  *ncell = total;
  *cells_out = dk.Current();
  *ids_out = dv.Current();
  return BAL_OK;
}

__global__ void k_body_mean(Dev S, const int32_t* __restrict__ body, const double* __restrict__ dir,
                            double* __restrict__ bsum) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < S.nv; v += gridDim.x * blockDim.x)
    atomic_add3(bsum, body[v], ld3(dir, v));
}
// order-preserving 64-bit image of a double (for atomic min / max)
__device__ inline unsigned long long ord(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
// per body: max |p_v - pbar_B| and the AABB of its vertices at x
__global__ void k_body_stats(Dev S, const int32_t* __restrict__ body, const double* __restrict__ x,
                             const double* __restrict__ dir, const double* __restrict__ bmean,
                             unsigned long long* __restrict__ stats) {   // [nb][7]
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < S.nv; v += gridDim.x * blockDim.x) {
    const int b = body[v];
    const d3 w = ld3(dir, v) - d3{bmean[3 * b], bmean[3 * b + 1], bmean[3 * b + 2]};
    unsigned long long* st = stats + 7 * (int64_t)b;
    atomicMax(st, ord(sqrt(dot(w, w))));
    const d3 p = ld3(x, v);
    atomicMin(st + 1, ord(p.x));
    atomicMin(st + 2, ord(p.y));
    atomicMin(st + 3, ord(p.z));
    atomicMax(st + 4, ord(p.x));
    atomicMax(st + 5, ord(p.y));
    atomicMax(st + 6, ord(p.z));
  }
}
__global__ void k_stats_init(unsigned long long* stats, int nb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 7 * nb; i += gridDim.x * blockDim.x) {
    const int k = i % 7;
    stats[i] = (k >= 1 && k <= 3) ? ~0ull : 0ull;
  }
}

__global__ void k_body_div(double* bsum, const double* __restrict__ inv_cnt, int nb) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    bsum[3 * b] *= inv_cnt[b];
    bsum[3 * b + 1] *= inv_cnt[b];
    bsum[3 * b + 2] *= inv_cnt[b];
  }
}
template <int NT>
__global__ void __launch_bounds__(NT) k_rsum(Dev S, Grid G, double* partials) {
  double m = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < S.nsv; i += gridDim.x * NT) m += vert_r(G, S.surf[i]);
  m = block_sum<double, NT>(m);
  if (threadIdx.x == 0) partials[blockIdx.x] = m;
}

// one grid pass appending to out (counter not reset here)
bal_status grid_pass(Scene& S, const double* x, Grid& G, Buf& out, int64_t cap,
                     unsigned long long* counter, cudaStream_t st) {
  G.inv_c = 1.0 / (2.0 * G.rmax + 1.5 * S.mean_edge);
  int64_t ncell = 0;
  uint64_t* cells = nullptr;
  int32_t* ids = nullptr;
  BAL_TRY(build_cells(S, x, 0, S.d.nf, G, &ncell, &cells, &ids, st));
  if (ncell > 0 && S.d.nsv > 0) {
    k_pt_query<<<grid_for(S.d.nsv), kThreads, 0, st>>>(S.d, x, G, cells, ids, ncell,
                                                        out.as<uint64_t>(), counter, cap);
    ::bal::note_launch();
    BAL_LAUNCH_CHECK();
  }
  BAL_TRY(build_cells(S, x, 1, S.d.ne, G, &ncell, &cells, &ids, st));
  if (ncell > 0) {
    k_ee_query<<<grid_for(S.d.ne), kThreads, 0, st>>>(S.d, x, G, cells, ids, ncell,
                                                       out.as<uint64_t>(), counter, cap);
    ::bal::note_launch();
    BAL_LAUNCH_CHECK();
  }
  return BAL_OK;
}

// runs the passes, growing `out` until the pairs fit, then sorts the keys
bal_status collect(Scene& S, const double* x, Grid* passes, int npass, Buf& out, Buf& alt,
                   int64_t* n, cudaStream_t st) {
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(S.scal + 63);
  int64_t cap = (int64_t)(out.cap / sizeof(uint64_t));
  if (cap < 1024) {
    BAL_TRY(buf_reserve(out, sizeof(uint64_t) * 1024));
    cap = (int64_t)(out.cap / sizeof(uint64_t));
  }
  unsigned long long found = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    BAL_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
    for (int k = 0; k < npass; ++k) BAL_TRY(grid_pass(S, x, passes[k], out, cap, counter, st));
    BAL_CUDA(cudaMemcpyAsync(&found, counter, sizeof(found), cudaMemcpyDeviceToHost, st));
    BAL_CUDA(cudaStreamSynchronize(st));
    if ((int64_t)found <= cap) break;
    if ((int64_t)found > S.pair_limit) {
      set_error("broad phase: %llu candidate pairs exceed pair_limit %lld", found,
                (long long)S.pair_limit);
      return BAL_ERR_CAPACITY;
    }
    BAL_TRY(buf_reserve(out, sizeof(uint64_t) * (found + found / 4 + 1024)));
    cap = (int64_t)(out.cap / sizeof(uint64_t));
  }
  *n = (int64_t)found;
  if (found > 1) {
    BAL_TRY(buf_reserve(alt, sizeof(uint64_t) * found));
    cub::DoubleBuffer<uint64_t> dk(out.as<uint64_t>(), alt.as<uint64_t>());
    size_t tmp = 0;
    BAL_CUDA(cub::DeviceRadixSort::SortKeys(nullptr, tmp, dk, (int64_t)found, 0, 64, st));
    BAL_TRY(buf_reserve(S.cub_tmp, tmp));
    BAL_CUDA(cub::DeviceRadixSort::SortKeys(S.cub_tmp.p, tmp, dk, (int64_t)found, 0, 64, st));
    if (dk.Current() != out.as<uint64_t>()) std::swap(out, alt);
  }
  return BAL_OK;
}

}  // namespace

bal_status find_candidates(Scene& S, const double* x, double r, Buf& out, Buf& alt, int64_t* n,
                           cudaStream_t st) {
  if (S.prm.broad_phase == BAL_BROAD_LBVH) return lbvh_candidates(S, x, nullptr, r, out, alt, n, st);
  Grid G{};
  G.mode = 0;
  G.half_r = 0.5 * r;
  G.rmax = 0.5 * r;   // (uniform radius)
  return collect(S, x, &G, 1, out, alt, n, st);
}

static inline double unord(unsigned long long u) {
  const unsigned long long v = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
  double d;
  std::memcpy(&d, &v, sizeof(d));
  return d;
}

bal_status find_candidates_motion(Scene& S, const double* x, const double* dir, Buf& out, Buf& alt,
                                  int64_t* n, cudaStream_t st) {
  // the LBVH form keeps the pairs whose swept boxes come within dhat: every pair
  // that can enter A during the step, and every pair the CCD bound can activate
  if (S.prm.broad_phase == BAL_BROAD_LBVH) return lbvh_candidates(S, x, dir, S.d.dhat, out, alt, n, st);
  const int nb = S.nbody;
  // per-body mean displacement of the step, deviation bound and AABB
  BAL_CUDA(cudaMemsetAsync(S.bmean, 0, sizeof(double) * 3 * nb, st));
  k_body_mean<<<grid_for(S.d.nv), kThreads, 0, st>>>(S.d, S.body, dir, S.bmean);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  k_body_div<<<grid_for(nb), kThreads, 0, st>>>(S.bmean, S.body_inv_cnt, nb);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  BAL_TRY(buf_reserve(S.bstats, sizeof(unsigned long long) * 7 * nb));
  unsigned long long* stats = S.bstats.as<unsigned long long>();
  k_stats_init<<<grid_for(7 * nb), kThreads, 0, st>>>(stats, nb);
  ::bal::note_launch();
  k_body_stats<<<grid_for(S.d.nv), kThreads, 0, st>>>(S.d, S.body, x, dir, S.bmean, stats);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  std::vector<double> pm(3 * nb);
  std::vector<unsigned long long> sh(7 * (size_t)nb);
  BAL_CUDA(cudaMemcpyAsync(pm.data(), S.bmean, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, st));
  BAL_CUDA(cudaMemcpyAsync(sh.data(), stats, sizeof(unsigned long long) * 7 * nb, cudaMemcpyDeviceToHost, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  // Bodies B, C can hold a pair with d < Delta/eta + dhat only if their boxes
  // are within (rho_B + rho_C + |pbar_B - pbar_C|)/eta + dhat; each body is then
  // inflated by half of the largest |pbar_B - pbar_C| over such C.
  const double eta = S.prm.step_bound, dh = S.d.dhat;
  std::vector<double> mot(nb, 0.0);
  if (nb <= 8192) {
    for (int b = 0; b < nb; ++b) {
      const unsigned long long* sb = &sh[7 * (size_t)b];
      for (int c = b + 1; c < nb; ++c) {
        const unsigned long long* sc = &sh[7 * (size_t)c];
        const double dx = pm[3 * b] - pm[3 * c], dy = pm[3 * b + 1] - pm[3 * c + 1],
                     dz = pm[3 * b + 2] - pm[3 * c + 2];
        const double m = std::sqrt(dx * dx + dy * dy + dz * dz);
        const double reach = (unord(sb[0]) + unord(sc[0]) + m) / eta + dh;
        double gap2 = 0.0;
        for (int k = 0; k < 3; ++k) {
          const double g = std::max(unord(sc[1 + k]) - unord(sb[4 + k]), unord(sb[1 + k]) - unord(sc[4 + k]));
          if (g > 0) gap2 += g * g;
        }
        if (gap2 > reach * reach) continue;
        mot[b] = std::max(mot[b], 0.5 * m);
        mot[c] = std::max(mot[c], 0.5 * m);
      }
    }
  } else {   // many bodies: |pbar_B - pbar_C| <= |pbar_B - q| + |pbar_C - q|, q = mean
    double q[3] = {0, 0, 0};
    for (int b = 0; b < nb; ++b)
      for (int k = 0; k < 3; ++k) q[k] += pm[3 * b + k] / nb;
    for (int b = 0; b < nb; ++b) {
      double s2 = 0;
      for (int k = 0; k < 3; ++k) s2 += (pm[3 * b + k] - q[k]) * (pm[3 * b + k] - q[k]);
      mot[b] = std::sqrt(s2);
    }
  }
  BAL_CUDA(cudaMemcpyAsync(S.bmot, mot.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st));
  Grid P[2];
  for (int k = 0; k < 2; ++k) {
    P[k] = Grid{};
    P[k].mode = 1 + k;
    P[k].dir = dir;
    P[k].bmean = S.bmean;
    P[k].bmot = S.bmot;
    P[k].body = S.body;
    P[k].eta = eta;
    P[k].base = 0.5 * dh;
    constexpr int NT = 256;
    k_rsum<NT><<<2 * kNumSM, NT, 0, st>>>(S.d, P[k], S.partials);
    ::bal::note_launch();
    BAL_LAUNCH_CHECK();
    BAL_TRY(finish_reduce(S, 2 * kNumSM, 15 + k, RED_SUM, st));
  }
  double rm[2];
  BAL_CUDA(cudaMemcpyAsync(rm, S.scal + 15, sizeof(rm), cudaMemcpyDeviceToHost, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  // rmax holds the mean surface radius: it only sets the cell size
  P[0].rmax = S.d.nsv ? rm[0] / S.d.nsv : dh;
  P[1].rmax = S.d.nsv ? rm[1] / S.d.nsv : dh;
  const int npass = nb > 1 ? 2 : 1;
  return collect(S, x, P, npass, out, alt, n, st);
}

}  // namespace bal
