// Arithmetic peak of the GPU for the roofline of the plain FP64 form (no
// counterpart in the paper).  The FP64 step is bound by the FP64 pipe, not by
// HBM, so its roofline needs the sustained fused multiply-add rate, measured
// here: every thread advances eight independent chains x <- x a + b (no
// memory traffic), on a grid of several blocks per SM, timed with CUDA events
// on the caller's stream.  The clocks are left as they are.
#include <cuda_runtime.h>

#include "cc_internal.h"

namespace {

constexpr int kChains = 8, kThreads = 256;

// target of the (never taken) store that keeps the chains from being removed
__device__ double g_sink[1];

template <typename T>
__global__ void k_fma_peak(int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int q = 0; q < kChains; q++) x[q] = (T)(threadIdx.x + q) * (T)1e-3;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int q = 0; q < kChains; q++) x[q] = fma(x[q], a, b);
  }
  T s = 0;
#pragma unroll
  for (int q = 0; q < kChains; q++) s += x[q];
  if (s == (T)-1) g_sink[0] = (double)s;  // the chains stay near 1: never taken
}

}  // namespace

extern "C" cc_status cc_fma_peak(int precision, int iters, void *stream, double *flops_per_s) {
  if (!flops_per_s || iters <= 0 || (precision != CC_FP64 && precision != CC_FP32)) return CC_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CC_ECUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CC_ECUDA;
  if (cudaPeekAtLastError() != cudaSuccess) return CC_ECUDA;  // an earlier call's error is not ours to clear
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = nsm * 8;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CC_ECUDA;
  auto launch = [&]() {
    if (precision == CC_FP64)
      k_fma_peak<double><<<blocks, kThreads, 0, st>>>(iters, 0.9999999, 1e-7);
    else
      k_fma_peak<float><<<blocks, kThreads, 0, st>>>(iters, 0.9999f, 1e-4f);
  };
  launch();  // warm-up
  cudaEventRecord(e0, st);
  launch();
  cudaEventRecord(e1, st);
  cc_status r = CC_OK;
  float ms = 0.0f;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
      cudaGetLastError() != cudaSuccess)
    r = CC_ECUDA;
  else
    *flops_per_s = 2.0 * kChains * (double)iters * blocks * kThreads / (ms * 1e-3);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return r;
}
