// Measured FP64 peak of the device (rt_fp64_peak, declared in include/rt.h).
// Not a step of the method: the denominator of the FP64 rooflines.  The
// chemistry (and every kernel of the FP64 sweep) is bound by GB300's FP64
// unit, so their fractions are taken against what a pure fused
// multiply-add stream achieves on this device, timed with CUDA events.
#include <cstdint>
#include <cstdio>

#include <cuda_runtime.h>

#include "../../include/rt.h"

namespace {

constexpr int kChains = 8;      // independent FMA chains per thread
constexpr int kThreads = 256;

thread_local char g_err[256];

rt_status fail(const char* what, cudaError_t e) {
  std::snprintf(g_err, sizeof g_err, "rt_fp64_peak: %s: %s", what, cudaGetErrorString(e));
  return RT_CUDA;
}

// kChains independent chains a <- a m + c per thread; m and c come from the
// host, so the compiler can neither fold nor shorten the chains.  Each
// iteration is kChains FP64 fused multiply-adds (2 FLOP each).
__global__ void __launch_bounds__(kThreads) k_dfma_stream(int iters, double m, double c, double* out) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int n = 0; n < iters; ++n) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" rt_status rt_fp64_peak(void* stream, int iters, int reps, double* tflops, double* ms_best) {
  if (!tflops || iters < 1 || iters > (1 << 20) || reps < 1 || reps > 100) {
    std::snprintf(g_err, sizeof g_err, "rt_fp64_peak: bad argument (iters 1..2^20, reps 1..100, tflops non-NULL)");
    return RT_INVALID_ARG;
  }
  int dev = 0, n_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail("no device", e);
  }
  // eight 256-thread blocks per SM: 64 warps, enough independent FP64 work
  // per scheduler to keep the pipe busy
  const int blocks = 8 * n_sm;
  cudaStream_t s = (cudaStream_t)stream;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = -1.0f;
  e = cudaMalloc(&out, sizeof(double) * (size_t)blocks * kThreads);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int r = 0; r <= reps && e == cudaSuccess; ++r) {   // r == 0: warm-up
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      k_dfma_stream<<<blocks, kThreads, 0, s>>>(iters, 0.999999999, 1e-9, out);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && (best < 0.0f || ms < best)) best = ms;
  }
  const cudaError_t err = e;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return fail("measurement", err);
  }
  const double flop = 2.0 * kChains * (double)iters * blocks * kThreads;
  *tflops = flop / (best * 1e-3) / 1e12;
  if (ms_best) *ms_best = best;
  return RT_OK;
}

extern "C" const char* rt_fp64_peak_last_error(void) { return g_err; }
