// Arithmetic-throughput probe: the FP64 (or FP32) fused multiply-add rate
// this GPU sustains on independent chains.  The FP64 kernels of this library
// are bound by that rate rather than by memory bandwidth, so it is the
// denominator of their roofline fraction; the benchmark measures it here
// beside the figure derived from the unit count and the clock.  (A
// measurement utility: the paper has no counterpart.)
#include <cuda_runtime.h>

#include "../../include/tdse.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;   // 2048 threads per SM: every issue slot has work
constexpr int kChains = 8;        // independent FMA chains per thread

// Written only if a chain reaches an impossible value: it keeps the chains
// live without a store per thread (and needs no allocation).
__device__ double g_probe_sink;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chains_kernel(T a0, T b, T c, int iters) {
  T v[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) v[k] = a0 + (T)(threadIdx.x * kChains + k) * (T)1e-7;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) v[k] = fma(v[k], b, c);   // fixed point c / (1 - b) = 1
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += v[k];
  if (s == (T)-1) g_probe_sink = (double)s;
}

template <typename T>
cudaError_t run(int sms, int iters, cudaStream_t st) {
  fma_chains_kernel<T><<<sms * kBlocksPerSM, kThreads, 0, st>>>((T)0.5, (T)0.999999, (T)1e-6, iters);
  return cudaGetLastError();
}

}  // namespace

extern "C" int tdse_fma_throughput(int fp64, double *flops_per_s, void *cuda_stream) {
  if (!flops_per_s) return TDSE_ERR_ARG;
  *flops_per_s = 0.0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return TDSE_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // about 20 ms per timed launch at the expected rates (FP64 ~1.2e12, FP32 ~7.5e13 flop/s)
  const int iters = fp64 ? 5000 : 300000;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return TDSE_ERR_CUDA;
  }
  cudaError_t e = fp64 ? run<double>(sms, iters / 10, st) : run<float>(sms, iters / 10, st);   // warm-up
  float best = 0.f;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(a, st);
    if (e == cudaSuccess) e = fp64 ? run<double>(sms, iters, st) : run<float>(sms, iters, st);
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess || !(best > 0.f)) return TDSE_ERR_CUDA;
  const double fmas = (double)sms * kBlocksPerSM * kThreads * kChains * (double)iters;
  *flops_per_s = 2.0 * fmas / (1e-3 * (double)best);
  return TDSE_OK;
}
