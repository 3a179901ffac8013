// FP64 FMA throughput of the device (measurement support, not in the paper):
// the ALU ceiling of the FP64 kernels of the path (element eigensystems,
// contact stencils, the FP64 PCG), which B300 runs at a small fraction of its
// FP32 rate. Every thread runs kChains independent FMA recurrences, so the
// FP64 pipe, not the dependency latency, bounds the kernel.
#include "scene.cuh"

namespace bal {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fma_probe(double a, double b, int iters, double* out) {
  double c[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) c[k] = 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) c[k] = fma(c[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += c[k];
  if (s == -1.0) out[blockIdx.x] = s;   // keeps the chains live; never true for these inputs
}

}  // namespace
}  // namespace bal

using namespace bal;

extern "C" bal_status bal_fp64_fma_rate(int32_t iters, double* tflops, void* stream) {
  if (iters <= 0 || !tflops) {
    set_error("bal_fp64_fma_rate: iters must be positive and tflops non-null");
    return BAL_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  BAL_CUDA(cudaGetDevice(&dev));
  BAL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = nsm * 8, threads = 256;
  double* sink = nullptr;
  BAL_CUDA(cudaMallocAsync(&sink, sizeof(double) * blocks, st));
  cudaEvent_t e0, e1;
  BAL_CUDA(cudaEventCreate(&e0));
  BAL_CUDA(cudaEventCreate(&e1));
  k_fma_probe<<<blocks, threads, 0, st>>>(0.9999999, 1e-7, iters, sink);   // warm-up
  BAL_CUDA(cudaEventRecord(e0, st));
  k_fma_probe<<<blocks, threads, 0, st>>>(0.9999999, 1e-7, iters, sink);
  BAL_CUDA(cudaEventRecord(e1, st));
  ::bal::note_launch(2);
  BAL_LAUNCH_CHECK();
  BAL_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  BAL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  BAL_CUDA(cudaEventDestroy(e0));
  BAL_CUDA(cudaEventDestroy(e1));
  BAL_CUDA(cudaFreeAsync(sink, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  const double flops = 2.0 * kChains * (double)iters * blocks * threads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return BAL_OK;
}
