// Shared device helpers for libbal: error plumbing, 3-vector math, and
// deterministic block reductions (fixed tree order).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/bal.h"

namespace bal {

// ---- host error plumbing ---------------------------------------------------
void set_error(const char* fmt, ...);
void note_launch(int n = 1);   // counts this library's kernel launches (bal_launch_count)
bal_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define BAL_CUDA(call)                                                               \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) return ::bal::cuda_fail(e_, #call, __FILE__, __LINE__);   \
  } while (0)

#define BAL_TRY(call)          \
  do {                         \
    bal_status s_ = (call);    \
    if (s_ != BAL_OK) return s_; \
  } while (0)

#define BAL_LAUNCH_CHECK() BAL_CUDA(cudaGetLastError())

constexpr int kThreads = 256;       // default CTA size
constexpr int kNumSM = 148;         // B300

inline int grid_for(int64_t n, int threads = kThreads, int cap = kNumSM * 16) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// ---- small vector math -------------------------------------------------------
struct d3 {
  double x, y, z;
};
__host__ __device__ inline d3 operator+(d3 a, d3 b) { return d3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__host__ __device__ inline d3 operator-(d3 a, d3 b) { return d3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__host__ __device__ inline d3 operator-(d3 a) { return d3{-a.x, -a.y, -a.z}; }
__host__ __device__ inline d3 operator*(double s, d3 a) { return d3{s * a.x, s * a.y, s * a.z}; }
__host__ __device__ inline double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ inline d3 cross(d3 a, d3 b) {
  return d3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ inline d3 ld3(const double* p, int64_t i) {
  return d3{p[3 * i], p[3 * i + 1], p[3 * i + 2]};
}
__device__ inline void st3(double* p, int64_t i, d3 v) {
  p[3 * i] = v.x;
  p[3 * i + 1] = v.y;
  p[3 * i + 2] = v.z;
}
__device__ inline void atomic_add3(double* p, int64_t i, d3 v) {
  atomicAdd(p + 3 * i, v.x);
  atomicAdd(p + 3 * i + 1, v.y);
  atomicAdd(p + 3 * i + 2, v.z);
}

// ---- block reductions (result valid in thread 0) -------------------------------
template <typename T>
__device__ inline T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ inline T warp_min(T v) {
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_down_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}
template <typename T>
__device__ inline T warp_max(T v) {
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_down_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}
template <typename T, int NT>
__device__ inline T block_sum(T v) {
  __shared__ T sh[NT / 32];
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  T r = T(0);
  if (w == 0) {
    r = (l < NT / 32) ? sh[l] : T(0);
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}
template <typename T, int NT>
__device__ inline T block_min(T v, T ident) {
  __shared__ T sh[NT / 32];
  v = warp_min(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  T r = ident;
  if (w == 0) {
    r = (l < NT / 32) ? sh[l] : ident;
    r = warp_min(r);
  }
  __syncthreads();
  return r;
}
template <typename T, int NT>
__device__ inline T block_max(T v, T ident) {
  __shared__ T sh[NT / 32];
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  T r = ident;
  if (w == 0) {
    r = (l < NT / 32) ? sh[l] : ident;
    r = warp_max(r);
  }
  __syncthreads();
  return r;
}

}  // namespace bal
