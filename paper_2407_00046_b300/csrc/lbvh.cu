// Linear BVH broad phase (Sec. 5.3): one tree over the surface triangles and
// one over the surface edges. Primitives are ordered along a Morton curve
// (64-bit keys: the 30-bit Morton code of the box centre in the high word, the
// primitive index in the low word, so keys are unique); the sorted keys define a
// binary radix tree (internal node i splits at the highest bit where its key
// range differs); node boxes are filled bottom-up, the second child to arrive
// at a node (an atomic counter per node) computing the union.
//
// Queries: every surface vertex against the triangle tree (PT), every edge
// against the edge tree (EE, pairs e < f sharing no vertex). A query box is the
// primitive's box, inflated by r, and, for a line-search query along x + t dir,
// the box of its positions at t = 0 and t = 1 (the primitive boxes are swept
// the same way). Two primitives whose (swept) boxes are farther than r apart on
// some axis can not come within r of each other. Output: the same sorted pair
// keys as the grid broad phase.
#include <cub/cub.cuh>

#include "scene.cuh"

namespace bal {

namespace {

struct Box {
  double lo[3], hi[3];
};

__device__ inline void box_add(Box& b, d3 p) {
  b.lo[0] = fmin(b.lo[0], p.x); b.lo[1] = fmin(b.lo[1], p.y); b.lo[2] = fmin(b.lo[2], p.z);
  b.hi[0] = fmax(b.hi[0], p.x); b.hi[1] = fmax(b.hi[1], p.y); b.hi[2] = fmax(b.hi[2], p.z);
}
__device__ inline Box box_empty() {
  return Box{{INFINITY, INFINITY, INFINITY}, {-INFINITY, -INFINITY, -INFINITY}};
}
// box of vertices v[0..k) at x and, if dir, at x + dir
__device__ inline Box prim_box(const double* __restrict__ x, const double* __restrict__ dir, const int* v, int k) {
  Box b = box_empty();
  for (int a = 0; a < k; ++a) {
    const d3 p = ld3(x, v[a]);
    box_add(b, p);
    if (dir) box_add(b, p + ld3(dir, v[a]));
  }
  return b;
}
__device__ inline bool overlap(const Box& a, const Box& b, double r) {
  return a.lo[0] <= b.hi[0] + r && b.lo[0] <= a.hi[0] + r && a.lo[1] <= b.hi[1] + r &&
         b.lo[1] <= a.hi[1] + r && a.lo[2] <= b.hi[2] + r && b.lo[2] <= a.hi[2] + r;
}
__device__ inline void store_box(double* __restrict__ B, int64_t i, const Box& b) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    B[6 * i + k] = b.lo[k];
    B[6 * i + 3 + k] = b.hi[k];
  }
}
__device__ inline Box load_box_cg(const double* B, int64_t i) {
  Box b;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    b.lo[k] = __ldcg(B + 6 * i + k);
    b.hi[k] = __ldcg(B + 6 * i + 3 + k);
  }
  return b;
}

// vertices of primitive i: kind 0 = triangle, 1 = edge
__device__ inline int prim_verts(const Dev& S, int kind, int i, int v[3]) {
  if (kind == 0) {
    v[0] = S.tris[3 * i]; v[1] = S.tris[3 * i + 1]; v[2] = S.tris[3 * i + 2];
    return 3;
  }
  v[0] = S.edges[2 * i]; v[1] = S.edges[2 * i + 1];
  return 2;
}

// order-preserving map of doubles to unsigned integers (for atomicMin / Max)
__device__ inline unsigned long long ord_bits(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__host__ __device__ inline double ord_value(unsigned long long u) {
  const unsigned long long v = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
  double d;
  memcpy(&d, &v, sizeof(d));
  return d;
}

// primitive boxes and the bounds of their centres
template <int NT>
__global__ void __launch_bounds__(NT) k_prim_boxes(Dev S, int kind, int n, const double* __restrict__ x,
                                                   const double* __restrict__ dir, double* __restrict__ pbox,
                                                   unsigned long long* bounds) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) {
    int v[3];
    const int k = prim_verts(S, kind, i, v);
    const Box b = prim_box(x, dir, v, k);
    store_box(pbox, i, b);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double c = 0.5 * (b.lo[a] + b.hi[a]);
      lo[a] = fmin(lo[a], c);
      hi[a] = fmax(hi[a], c);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double l = block_min<double, NT>(lo[a], INFINITY);
    const double h = block_max<double, NT>(hi[a], -INFINITY);
    if (threadIdx.x == 0 && l <= h) {
      atomicMin(bounds + a, ord_bits(l));
      atomicMax(bounds + 3 + a, ord_bits(h));
    }
  }
}

__device__ inline unsigned int spread10(unsigned int v) {   // 10 bits -> every third bit
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
__global__ void k_morton(int n, const double* __restrict__ pbox, const unsigned long long* __restrict__ bounds,
                         uint64_t* __restrict__ keys) {
  double lo[3], ext[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = ord_value(bounds[a]);
    ext[a] = ord_value(bounds[3 + a]) - lo[a];
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    unsigned int q[3];
    for (int a = 0; a < 3; ++a) {
      const double c = 0.5 * (pbox[6 * (int64_t)i + a] + pbox[6 * (int64_t)i + 3 + a]);
      const double u = ext[a] > 0.0 ? (c - lo[a]) / ext[a] : 0.0;
      q[a] = (unsigned int)fmin(fmax(u * 1024.0, 0.0), 1023.0);
    }
    const unsigned int m = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    keys[i] = ((uint64_t)m << 32) | (uint32_t)i;
  }
}

// length of the common prefix of keys i and j (-1 outside [0, n))
__device__ inline int delta(const uint64_t* __restrict__ k, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  return __clzll((long long)(k[i] ^ k[j]));
}

// Internal node i covers a contiguous key range [min(i, j), max(i, j)] that
// starts or ends at i; it splits where the common prefix of the range ends.
// Nodes: internal 0 .. n-2 (0 the root), leaf l at n-1+l; child and parent
// arrays use that numbering.
__global__ void k_radix_tree(int n, const uint64_t* __restrict__ k, int2* __restrict__ child,
                             int* __restrict__ parent) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n - 1; i += gridDim.x * blockDim.x) {
    const int d = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta(k, n, i, i - d);
    int lmax = 2;
    while (delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
      if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = delta(k, n, i, j);
    int s = 0;
    for (int t = (l + 1) >> 1;; t = (t + 1) >> 1) {
      if (delta(k, n, i, i + (s + t) * d) > dnode) s += t;
      if (t == 1) break;
    }
    const int g = i + s * d + (d < 0 ? -1 : 0);
    const int left = (min(i, j) == g) ? (n - 1 + g) : g;
    const int right = (max(i, j) == g + 1) ? (n - 1 + g + 1) : g + 1;
    child[i] = make_int2(left, right);
    parent[left] = i;
    parent[right] = i;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) parent[0] = -1;
}

// leaf boxes in key order, then bottom-up unions
__global__ void k_leaf_boxes(int n, const uint64_t* __restrict__ k, const double* __restrict__ pbox,
                             double* __restrict__ nbox, int* __restrict__ prim) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
    const int p = (int)(uint32_t)k[l];
    prim[l] = p;
    for (int a = 0; a < 6; ++a) nbox[6 * (int64_t)(n - 1 + l) + a] = pbox[6 * (int64_t)p + a];
  }
}
__global__ void k_refit(int n, const int* __restrict__ parent, const int2* __restrict__ child,
                        double* nbox, unsigned int* __restrict__ arrivals) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
    int node = n > 1 ? parent[n - 1 + l] : -1;
    for (int depth = 0; node >= 0 && depth < 2 * n; ++depth) {
      __threadfence();   // this thread's child box is visible before it arrives
      if (atomicAdd(arrivals + node, 1u) == 0) break;   // first child: the other one finishes the node
      const int2 c = child[node];
      const Box a = load_box_cg(nbox, c.x), b = load_box_cg(nbox, c.y);
      Box u;
      for (int q = 0; q < 3; ++q) {
        u.lo[q] = fmin(a.lo[q], b.lo[q]);
        u.hi[q] = fmax(a.hi[q], b.hi[q]);
      }
      store_box(nbox, node, u);
      node = parent[node];
    }
  }
}

constexpr int kStack = 64;   // a root-to-leaf path splits at strictly later key bits: depth <= 64

// PT: surface vertex queries against the triangle tree; EE: edge queries
// against the edge tree (the tree and queries of the same kind)
__global__ void k_tree_query(Dev S, int kind, int nq, int ntree, const double* __restrict__ x,
                             const double* __restrict__ dir, double r, const double* __restrict__ nbox,
                             const int2* __restrict__ child, const int* __restrict__ prim,
                             uint64_t* __restrict__ out, unsigned long long* counter, int64_t cap,
                             unsigned int* overflow) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    int qv[3];
    int nqv;
    if (kind == 0) {
      qv[0] = S.surf[q];
      nqv = 1;
    } else {
      nqv = prim_verts(S, 1, q, qv);
    }
    const Box qb = prim_box(x, dir, qv, nqv);
    int stack[kStack];
    int sp = 0;
    stack[sp++] = ntree > 1 ? 0 : 0;   // root (the lone leaf is node 0 when ntree == 1)
    while (sp > 0) {
      const int node = stack[--sp];
      Box b;
      for (int a = 0; a < 3; ++a) {
        b.lo[a] = nbox[6 * (int64_t)node + a];
        b.hi[a] = nbox[6 * (int64_t)node + 3 + a];
      }
      if (!overlap(qb, b, r)) continue;
      if (node >= ntree - 1) {   // leaf
        const int p = prim[node - (ntree - 1)];
        int pv[3];
        const int npv = prim_verts(S, kind == 0 ? 0 : 1, p, pv);
        bool shared = false;
        for (int a = 0; a < nqv; ++a)
          for (int b2 = 0; b2 < npv; ++b2) shared |= qv[a] == pv[b2];
        if (shared) continue;
        if (kind == 1 && !(q < p)) continue;
        const uint64_t key = kind == 0 ? pair_key(0, (uint32_t)qv[0], (uint32_t)p) : pair_key(1, (uint32_t)q, (uint32_t)p);
        const unsigned long long slot = atomicAdd(counter, 1ull);
        if ((int64_t)slot < cap) out[slot] = key;
        continue;
      }
      if (sp + 2 > kStack) {
        atomicAdd(overflow, 1u);
        break;
      }
      const int2 c = child[node];
      stack[sp++] = c.x;
      stack[sp++] = c.y;
    }
  }
}

struct Tree {
  int n = 0;
  double* nbox = nullptr;
  int2* child = nullptr;
  int* prim = nullptr;
};

// builds the tree of kind (0 triangles, 1 edges) over boxes at x (swept along dir)
bal_status build_tree(Scene& S, int kind, const double* x, const double* dir, Tree* T, cudaStream_t st) {
  const int n = kind == 0 ? S.d.nf : S.d.ne;
  T->n = n;
  if (n == 0) return BAL_OK;
  const int nn = 2 * n - 1;
  BAL_TRY(buf_reserve(S.lb_pbox, sizeof(double) * 6 * (size_t)n));
  BAL_TRY(buf_reserve(S.lb_nbox, sizeof(double) * 6 * (size_t)nn));
  BAL_TRY(buf_reserve(S.lb_keys, sizeof(uint64_t) * (size_t)n));
  BAL_TRY(buf_reserve(S.lb_keys_alt, sizeof(uint64_t) * (size_t)n));
  BAL_TRY(buf_reserve(S.lb_child, sizeof(int2) * (size_t)std::max(n - 1, 1)));
  BAL_TRY(buf_reserve(S.lb_parent, sizeof(int) * (size_t)nn));
  BAL_TRY(buf_reserve(S.lb_prim, sizeof(int) * (size_t)n));
  BAL_TRY(buf_reserve(S.lb_arrivals, sizeof(unsigned int) * (size_t)std::max(n - 1, 1)));
  BAL_TRY(buf_reserve(S.lb_bounds, sizeof(unsigned long long) * 6));
  unsigned long long init[6];
  for (int a = 0; a < 3; ++a) {
    init[a] = ~0ull;       // min of ordered bits
    init[3 + a] = 0ull;    // max
  }
  BAL_CUDA(cudaMemcpyAsync(S.lb_bounds.p, init, sizeof(init), cudaMemcpyHostToDevice, st));
  k_prim_boxes<kThreads><<<grid_for(n), kThreads, 0, st>>>(S.d, kind, n, x, dir, S.lb_pbox.as<double>(),
                                                           S.lb_bounds.as<unsigned long long>());
  ::bal::note_launch();
  k_morton<<<grid_for(n), kThreads, 0, st>>>(n, S.lb_pbox.as<double>(), S.lb_bounds.as<unsigned long long>(),
                                            S.lb_keys.as<uint64_t>());
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  cub::DoubleBuffer<uint64_t> dk(S.lb_keys.as<uint64_t>(), S.lb_keys_alt.as<uint64_t>());
  size_t tmp = 0;
  BAL_CUDA(cub::DeviceRadixSort::SortKeys(nullptr, tmp, dk, n, 0, 64, st));
  BAL_TRY(buf_reserve(S.cub_tmp, tmp));
  BAL_CUDA(cub::DeviceRadixSort::SortKeys(S.cub_tmp.p, tmp, dk, n, 0, 64, st));
  const uint64_t* keys = dk.Current();
  k_leaf_boxes<<<grid_for(n), kThreads, 0, st>>>(n, keys, S.lb_pbox.as<double>(), S.lb_nbox.as<double>(),
                                                 S.lb_prim.as<int>());
  ::bal::note_launch();
  if (n > 1) {
    k_radix_tree<<<grid_for(n - 1), kThreads, 0, st>>>(n, keys, S.lb_child.as<int2>(), S.lb_parent.as<int>());
    ::bal::note_launch();
    BAL_CUDA(cudaMemsetAsync(S.lb_arrivals.p, 0, sizeof(unsigned int) * (size_t)(n - 1), st));
    k_refit<<<grid_for(n), kThreads, 0, st>>>(n, S.lb_parent.as<int>(), S.lb_child.as<int2>(),
                                              S.lb_nbox.as<double>(), S.lb_arrivals.as<unsigned int>());
    ::bal::note_launch();
  }
  BAL_LAUNCH_CHECK();
  T->nbox = S.lb_nbox.as<double>();
  T->child = S.lb_child.as<int2>();
  T->prim = S.lb_prim.as<int>();
  return BAL_OK;
}

bal_status query_pass(Scene& S, const double* x, const double* dir, double r, Buf& out, int64_t cap,
                      unsigned long long* counter, unsigned int* overflow, cudaStream_t st) {
  for (int kind = 0; kind < 2; ++kind) {
    Tree T;
    BAL_TRY(build_tree(S, kind, x, dir, &T, st));
    const int nq = kind == 0 ? S.d.nsv : S.d.ne;
    if (T.n == 0 || nq == 0) continue;
    k_tree_query<<<grid_for(nq), kThreads, 0, st>>>(S.d, kind, nq, T.n, x, dir, r, T.nbox, T.child, T.prim,
                                                    out.as<uint64_t>(), counter, cap, overflow);
    ::bal::note_launch();
    BAL_LAUNCH_CHECK();
  }
  return BAL_OK;
}

}  // namespace

bal_status lbvh_candidates(Scene& S, const double* x, const double* dir, double r, Buf& out, Buf& alt,
                           int64_t* n, cudaStream_t st) {
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(S.scal + 63);
  unsigned int* overflow = reinterpret_cast<unsigned int*>(S.scal + 60);
  int64_t cap = (int64_t)(out.cap / sizeof(uint64_t));
  if (cap < 1024) {
    BAL_TRY(buf_reserve(out, sizeof(uint64_t) * 1024));
    cap = (int64_t)(out.cap / sizeof(uint64_t));
  }
  unsigned long long found = 0;
  unsigned int ovf = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    BAL_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
    BAL_CUDA(cudaMemsetAsync(overflow, 0, sizeof(unsigned int), st));
    BAL_TRY(query_pass(S, x, dir, r, out, cap, counter, overflow, st));
    BAL_CUDA(cudaMemcpyAsync(&found, counter, sizeof(found), cudaMemcpyDeviceToHost, st));
    BAL_CUDA(cudaMemcpyAsync(&ovf, overflow, sizeof(ovf), cudaMemcpyDeviceToHost, st));
    BAL_CUDA(cudaStreamSynchronize(st));
    if (ovf) {
      set_error("lbvh: traversal stack overflow in %u queries", ovf);
      return BAL_ERR_CAPACITY;
    }
    if ((int64_t)found <= cap) break;
    if ((int64_t)found > S.pair_limit) {
      set_error("lbvh: %llu candidate pairs exceed pair_limit %lld", found, (long long)S.pair_limit);
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

}  // namespace bal
