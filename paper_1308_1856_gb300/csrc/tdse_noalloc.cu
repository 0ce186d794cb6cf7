// tdse_observables_noalloc: the observables reduction without any allocation.
//
// Who needs this: code that runs where cudaMalloc is not an option -- for
// example a plugin or callback invoked inside someone else's CUDA-graph
// capture or real-time loop (an allocation there would synchronise the device
// or break the capture), or an embedding that forbids the library from
// owning device memory.  Such a caller cannot create a tdse handle (which
// allocates its tables and scratch), but it can still hand over a state it
// already holds on the device and a device buffer for the results.
//
// How: the per-block partial sums live in one file-scope __device__ array of
// fixed size instead of in memory the library allocates.  Every GPU that
// loads this library reserves that array until the process exits.  All calls
// share it, so two calls whose kernels overlap on the GPU (different streams,
// no ordering between them) race and give wrong results; calls issued on one
// stream, or otherwise ordered, are fine.  The array keeps the last call's
// contents; the only part that must start at zero (the arrival counter) is
// cleared before each launch.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/tdse.h"

namespace {

constexpr int kThreads = 256;
constexpr int kQ = 5;          // quantities per block: |f|^2, inside r_b, dipole, overlap re/im
constexpr int kMaxBx = 8;      // blocks per partial wave
constexpr int kMaxRows = TDSE_NOALLOC_MAX_LMAX + 1;
constexpr int kScratchDoubles = kQ * kMaxBx * kMaxRows;

struct NoallocScratch {
  double partial[kScratchDoubles];
  unsigned int ticket;
  unsigned int pad[63];
};

// The scratch itself (about 80 KB): block partials and the arrival counter.
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// Device address of g_noalloc_scratch per device, looked up once per device.
constexpr int kMaxDevices = 64;
NoallocScratch *g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v, double *sh) {
  const int tid = threadIdx.x;
  v = warp_sum(v);
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    double s = (tid < kThreads / 32) ? sh[tid] : 0.0;
    s = warp_sum(s);
    if (tid == 0) sh[kThreads / 32] = s;
  }
  __syncthreads();
  const double r = sh[kThreads / 32];
  __syncthreads();
  return r;
}

// Same sums as the handle-based observables (Sec. 4 of arXiv 1308.1856, every
// integral as dr times a sum over grid points), with r_j and kappa_l formed
// in the kernel so that no table is needed.
__global__ void __launch_bounds__(kThreads)
    observables_noalloc_kernel(const double2 *__restrict__ psi, const double2 *__restrict__ ref0,
                               int N, int L, double dr, double offset, double r_b,
                               NoallocScratch *scratch, double *out) {
  __shared__ double sh[kThreads / 32 + 1];
  __shared__ unsigned s_last;
  const int l = blockIdx.y;
  const int nbx = gridDim.x;
  double q[kQ] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < N; i += nbx * kThreads) {
    const size_t idx = (size_t)l * N + i;
    const double2 f = psi[idx];
    const double a = __fma_rn(f.x, f.x, __dmul_rn(f.y, f.y));
    // rounded as the host's grid table (multiply, then add; no fused step), so
    // that r_j <= r_b decides the same way when r_b falls on a grid point
    const double r = __dadd_rn(__dmul_rn((double)(i + 1), dr), offset);
    q[0] += a;
    if (r <= r_b) q[1] += a;
    if (l < L) {
      const double2 g = psi[idx + N];
      q[2] = __fma_rn(r, __fma_rn(f.x, g.x, __dmul_rn(f.y, g.y)), q[2]);
    }
    if (l == 0 && ref0) {
      const double2 c = ref0[i];
      q[3] += __fma_rn(c.x, f.x, __dmul_rn(c.y, f.y));
      q[4] += __fma_rn(c.x, f.y, __dmul_rn(-c.y, f.x));
    }
  }
  const size_t nb = (size_t)nbx * (L + 1);
  const size_t bid = (size_t)l * nbx + blockIdx.x;
  for (int k = 0; k < kQ; ++k) {
    const double b = block_sum(q[k], sh);
    if (threadIdx.x == 0) scratch->partial[(size_t)k * nb + bid] = b;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(&scratch->ticket, 1u) == nb - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double norm_part = 0.0, inside_part = 0.0, dip_part = 0.0;
  for (int row = threadIdx.x; row <= L; row += kThreads) {
    double p0 = 0.0, p1 = 0.0, p2 = 0.0;
    for (int bx = 0; bx < nbx; ++bx) {
      const size_t o = (size_t)row * nbx + bx;
      p0 += __ldcg(&scratch->partial[0 * nb + o]);
      p1 += __ldcg(&scratch->partial[1 * nb + o]);
      p2 += __ldcg(&scratch->partial[2 * nb + o]);
    }
    out[4 + row] = dr * p0;
    norm_part += p0;
    inside_part += p1;
    if (row < L) {
      const double ll = (double)(row + 1) * (double)(row + 1);
      dip_part += 2.0 * sqrt(ll / (4.0 * ll - 1.0)) * dr * p2;
    }
  }
  const double norm = block_sum(norm_part, sh);
  const double inside = block_sum(inside_part, sh);
  const double dip = block_sum(dip_part, sh);
  if (threadIdx.x == 0) {
    double ore = 0.0, oim = 0.0;
    for (int bx = 0; bx < nbx; ++bx) {
      ore += __ldcg(&scratch->partial[3 * nb + bx]);
      oim += __ldcg(&scratch->partial[4 * nb + bx]);
    }
    ore *= dr;
    oim *= dr;
    out[0] = dr * norm;
    out[1] = dip;
    out[2] = 1.0 - dr * inside;
    out[3] = ore * ore + oim * oim;
    // a state holding Inf or NaN makes the norm sum non-finite
    out[L + 5] = isfinite(norm) ? 0.0 : 1.0;
    scratch->ticket = 0u;
  }
}

// Device address of the scratch on the current device (looked up on first use).
cudaError_t scratch_for_current_device(NoallocScratch **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<NoallocScratch *>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int tdse_observables_noalloc(int N, double dr, int lmax, double offset, double r_b,
                                        const void *psi_dev, const void *ref0_dev, double *out_dev,
                                        void *cuda_stream) {
  if (N < 1 || lmax < 0 || !(dr > 0.0) || !std::isfinite(offset) || std::isnan(r_b))
    return TDSE_ERR_ARG;
  if (lmax > TDSE_NOALLOC_MAX_LMAX) return TDSE_ERR_ARG;   // beyond the fixed scratch
  if (!(dr + offset > 0.0)) return TDSE_ERR_ARG;
  if (!psi_dev || !out_dev || ((uintptr_t)psi_dev & 15) || ((uintptr_t)ref0_dev & 15) ||
      ((uintptr_t)out_dev & 7))
    return TDSE_ERR_ARG;
  NoallocScratch *scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return TDSE_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // the arrival counter must start at zero; everything else is written before it is read
  e = cudaMemsetAsync(&scratch->ticket, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return TDSE_ERR_CUDA;
  const int per_row = (N + kThreads - 1) / kThreads;
  const int nbx = per_row < kMaxBx ? per_row : kMaxBx;
  const dim3 grid(nbx, lmax + 1);
  observables_noalloc_kernel<<<grid, kThreads, 0, st>>>(
      static_cast<const double2 *>(psi_dev), static_cast<const double2 *>(ref0_dev), N, lmax, dr,
      offset, r_b, scratch, out_dev);
  return cudaGetLastError() == cudaSuccess ? TDSE_OK : TDSE_ERR_CUDA;
}
