// Allocation-free mass sum.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool, a host application that reserves all device memory
// up front, or a process that must not allocate once it has started. This
// entry point computes the same compensated mass sum as cc_diagnostics from
// device buffers the caller already owns, and keeps its own scratch (one
// partial sum per block) in a fixed-size array in the library's device
// memory, so it allocates nothing.
#include <cuda_runtime.h>

#include <math.h>

#include <stdio.h>

#include <mutex>

#include "cc_internal.h"

namespace {

constexpr int kThreads = 256;

// Scratch: one (sum, compensation) pair per partial.  Every GPU that loads the
// library holds this array until the process exits.
static __device__ __align__(256) double g_parts[2 * CC_NOALLOC_MAX_PARTS];

// In host code g_parts names a host-side stand-in, not device memory: the
// device address is looked up once per device with that device current.
constexpr int kMaxDevices = 128;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {nullptr};

thread_local char g_msg[256];  // fixed buffer: error reporting allocates nothing either

// Each block writes its own slot; the final kernel reads exactly the slots
// written by the same call, so nothing needs clearing between calls.  The
// per-thread sums and the warp-shuffle trees are those of cc_diagnostics, so
// with 256 partials (its block count) the two give the same bits.
template <typename T>
__global__ void k_mass_parts(const T *__restrict__ rho, const double *__restrict__ vol, long long n,
                             double *__restrict__ parts) {
  cc::NSum<T> acc{0, 0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    acc.add((T)vol[i] * rho[i]);
  __shared__ cc::CSum sh[kThreads / 32];
  const cc::CSum b = cc::block_csum<kThreads>(cc::CSum{(double)acc.s, (double)acc.c}, sh);
  if (threadIdx.x == 0) {
    parts[2 * blockIdx.x] = b.s;
    parts[2 * blockIdx.x + 1] = b.c;
  }
}

__global__ void k_mass_final(const double *__restrict__ parts, int nparts, double *__restrict__ out) {
  cc::CSum b{0.0, 0.0};
  for (int p = threadIdx.x; p < nparts; p += kThreads) b = cc::csum_add(b, cc::CSum{parts[2 * p], parts[2 * p + 1]});
  __shared__ cc::CSum sh[kThreads / 32];
  b = cc::block_csum<kThreads>(b, sh);
  if (threadIdx.x == 0) {
    out[0] = b.s + b.c;
    out[1] = b.c;
  }
}

cc_status fail(cc_status s, const char *what, const char *detail = "") {
  snprintf(g_msg, sizeof(g_msg), "%s%s", what, detail);
  return s;
}

}  // namespace

extern "C" const char *cc_noalloc_last_error(void) { return g_msg; }

extern "C" cc_status cc_mass_sum_noalloc(const void *rho_prime, int precision, const double *volume, long long n,
                                         int nparts, double *out, void *stream) {
  if (!rho_prime || !volume || !out) return fail(CC_EINVAL, "null device pointer");
  if (precision != CC_FP64 && precision != CC_FP32) return fail(CC_EINVAL, "precision must be CC_FP64 or CC_FP32");
  if (n < 0) return fail(CC_EINVAL, "negative element count");
  if (nparts < 1 || nparts > CC_NOALLOC_MAX_PARTS)
    return fail(CC_EINVAL, "nparts must be in 1..1024 (the fixed scratch holds that many partial sums)");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(CC_ECUDA, "cudaGetDevice: ", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(CC_EINVAL, "device ordinal out of range");
  double *parts = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_parts);
      if (e != cudaSuccess || !p)
        return fail(CC_ECUDA, "cudaGetSymbolAddress: ", cudaGetErrorString(e));
      g_addr[dev] = (double *)p;
    }
    parts = g_addr[dev];
  }
  // an error left by an earlier, unrelated launch is reported, not cleared
  // (it belongs to its caller), and nothing is launched on top of it
  e = cudaPeekAtLastError();
  if (e != cudaSuccess) return fail(CC_ECUDA, "a CUDA error from an earlier call is pending: ", cudaGetErrorString(e));
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == CC_FP64)
    k_mass_parts<double><<<nparts, kThreads, 0, st>>>((const double *)rho_prime, volume, n, parts);
  else
    k_mass_parts<float><<<nparts, kThreads, 0, st>>>((const float *)rho_prime, volume, n, parts);
  k_mass_final<<<1, kThreads, 0, st>>>(parts, nparts, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CC_ECUDA, "launch: ", cudaGetErrorString(e));
  return CC_OK;
}
