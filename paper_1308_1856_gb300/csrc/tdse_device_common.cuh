// Device helpers shared by the FP64 and mixed-precision kernels: the
// persistent-grid work split and the deterministic grid reductions.
#pragma once

#include <cuda_runtime.h>

#include "tdse_internal.cuh"

namespace tdse_dev {
namespace common {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum (fixed shuffle tree + fixed warp order); the result
// is valid in every thread.  `sh` needs blockDim/32 + 1 doubles.
__device__ __forceinline__ double block_sum(double v, double *sh) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nthreads = blockDim.x * blockDim.y;
  v = warp_sum(v);
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    // the tree of warp_sum over the nw warp sums, without the levels whose
    // partner lanes hold only zeros (adding them changes no value)
    const int nw = nthreads >> 5;
    double s = (tid < nw) ? sh[tid] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      if (o < nw) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (tid == 0) sh[nw] = s;
  }
  __syncthreads();
  const double r = sh[nthreads >> 5];
  __syncthreads();
  return r;
}

// Called by every thread of the last block: fixed-order sum of all partials.
// Each thread first issues all its loads (independent, so their latencies
// overlap) and then adds them in index order.
constexpr int kMaxPartialsPerThread = 16;
__device__ __forceinline__ double reduce_partials(Reduction *red, unsigned nparts, double *sh) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nthreads = blockDim.x * blockDim.y;
  __threadfence();
  double v[kMaxPartialsPerThread];
#pragma unroll
  for (int r = 0; r < kMaxPartialsPerThread; ++r) {
    const unsigned k = tid + (unsigned)r * nthreads;
    v[r] = (k < nparts) ? __ldcg(&red->partial[k]) : 0.0;
  }
  double s = 0.0;
#pragma unroll
  for (int r = 0; r < kMaxPartialsPerThread; ++r) s += v[r];
  s = block_sum(s, sh);
  if (tid == 0) red->ticket = 0u;
  return s;
}

// Global warp index and warp count of a 1-D persistent launch.
// Running sum of FP32 terms held as an unevaluated pair s + c: every addition
// is error-free (Knuth's TwoSum), so the pair keeps about twice the FP32
// precision and a long run of terms needs no FP64 arithmetic until value().
// (FP64 instructions, conversions included, issue at a small fraction of the
// FP32 rate on this part.)
struct PairSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = __fadd_rn(s, x);
    const float z = __fsub_rn(t, s);
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z)));
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

__device__ __forceinline__ int warp_id() { return blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); }
__device__ __forceinline__ int warp_count() { return gridDim.x * (blockDim.x >> 5); }

// Range [s0, s1) of `total` (< 2^32) work items owned by warp w of the W warps:
// q = total / W items each, one more for the first total - q W warps.  Only a
// 32-bit division: a 64-bit integer division compiles to FP64 arithmetic,
// which issues at 1/64 of the FP32 rate on this part.
__device__ __forceinline__ void warp_range(long long total, long long &s0, long long &s1) {
  const unsigned W = (unsigned)warp_count(), w = (unsigned)warp_id();
  const unsigned T = (unsigned)total;
  const unsigned q = T / W, r = T - q * W;
  s0 = (long long)w * q + (w < r ? w : r);
  s1 = s0 + q + (w < r ? 1u : 0u);
}

// Sum v over the block (fixed shuffle tree and warp order), store it as this
// block's partial and report whether this block is the last to finish.  The
// last block then adds all block partials in block order, so the result does
// not depend on timing.
__device__ __forceinline__ bool publish_block_partial(double v, Reduction *red, double *sh) {
  __shared__ unsigned s_last;
  const double b = block_sum(v, sh);
  if (threadIdx.x == 0) {
    red->partial[blockIdx.x] = b;
    __threadfence();
    const unsigned t = atomicAdd(&red->ticket, 1u);
    s_last = (t == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  return s_last != 0;
}

}  // namespace common
}  // namespace tdse_dev
