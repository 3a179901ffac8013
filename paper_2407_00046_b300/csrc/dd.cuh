// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers (|lo| <= ulp(hi)/2 after normalisation), a ~47-bit significand in
// FP32 registers. B300 runs FP32 about 58x faster than FP64, so the PCG
// recurrences in this form are bound by memory, not by the FP64 pipe.
//
// Built from the error-free transformations TwoSum (Knuth, TAOCP vol. 2,
// Sec. 4.2.2: s + e = a + b exactly) and TwoProduct with a fused multiply-add
// (the rounding error of a*b is fma(a, b, -a*b) exactly; Dekker 1971 gives the
// split form). Addition is the "sloppy" double-double sum: its error is below
// ~2^-47 (|a| + |b|), the same form as the error of one FP64 add scaled by 2^6.
// Every step uses round-to-nearest intrinsics, which the compiler neither
// contracts nor reorders.
#pragma once
#include <cuda_runtime.h>

namespace bal {

struct __align__(8) dd {
  float hi, lo;
};

__host__ __device__ inline dd dd_from(double x) {
  const float h = (float)x;
  return dd{h, (float)(x - (double)h)};
}
__host__ __device__ inline double dd_to(dd a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ dd dd_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dd{s, e};
}
// exact when the exponent of a is not below that of b
__device__ __forceinline__ dd dd_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dd{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  const dd s = dd_two_sum(a.hi, b.hi);
  return dd_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }
// a*b: exact product of the high parts plus the two cross terms (lo*lo dropped)
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dd_fast_two_sum(p, e);
}
// acc + a*b with one normalisation
__device__ __forceinline__ dd dd_fma(dd a, dd b, dd acc) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const dd s = dd_two_sum(acc.hi, p);
  return dd_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(acc.lo, e)));
}

struct dd3 {
  dd x, y, z;
};
__device__ __forceinline__ dd3 dd3_ld(const dd* __restrict__ p, int64_t i) {
  return dd3{p[3 * i], p[3 * i + 1], p[3 * i + 2]};
}
__device__ __forceinline__ void dd3_st(dd* __restrict__ p, int64_t i, dd3 v) {
  p[3 * i] = v.x;
  p[3 * i + 1] = v.y;
  p[3 * i + 2] = v.z;
}
__device__ __forceinline__ dd3 dd3_add(dd3 a, dd3 b) {
  return dd3{dd_add(a.x, b.x), dd_add(a.y, b.y), dd_add(a.z, b.z)};
}
// b + s a
__device__ __forceinline__ dd3 dd3_axpy(dd s, dd3 a, dd3 b) {
  return dd3{dd_fma(s, a.x, b.x), dd_fma(s, a.y, b.y), dd_fma(s, a.z, b.z)};
}
__device__ __forceinline__ dd dd3_dot(dd3 a, dd3 b) {
  return dd_fma(a.z, b.z, dd_fma(a.y, b.y, dd_mul(a.x, b.x)));
}
// B v and B^T v for a row-major 3x3 block
__device__ __forceinline__ dd3 dd3_mv(const dd* __restrict__ B, dd3 v) {
  dd b[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) b[k] = B[k];
  return dd3{dd_fma(b[2], v.z, dd_fma(b[1], v.y, dd_mul(b[0], v.x))),
             dd_fma(b[5], v.z, dd_fma(b[4], v.y, dd_mul(b[3], v.x))),
             dd_fma(b[8], v.z, dd_fma(b[7], v.y, dd_mul(b[6], v.x)))};
}
__device__ __forceinline__ dd3 dd3_mtv(const dd* __restrict__ B, dd3 v) {
  dd b[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) b[k] = B[k];
  return dd3{dd_fma(b[6], v.z, dd_fma(b[3], v.y, dd_mul(b[0], v.x))),
             dd_fma(b[7], v.z, dd_fma(b[4], v.y, dd_mul(b[1], v.x))),
             dd_fma(b[8], v.z, dd_fma(b[5], v.y, dd_mul(b[2], v.x)))};
}

// block sum of a double-float (fixed tree order); result valid in thread 0
template <int NT>
__device__ inline dd dd_block_sum(dd v) {
  __shared__ dd sh[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const dd w{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
    v = dd_add(v, w);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  dd r{0.f, 0.f};
  if (w == 0) {
    r = (l < NT / 32) ? sh[l] : dd{0.f, 0.f};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const dd u{__shfl_down_sync(0xffffffffu, r.hi, o), __shfl_down_sync(0xffffffffu, r.lo, o)};
      r = dd_add(r, u);
    }
  }
  __syncthreads();
  return r;
}

}  // namespace bal
