// Every Lanczos step of a tdse_propagate call in one cooperative launch (FP64,
// length gauge), for grids too large for one thread-block cluster.
//
// The multi-launch path (Appendix "Lanczos methods" of arXiv 1308.1856: per
// iteration j a stencil phase A, z = sigma_j H U_j - ratio_j U_{j-1} with
// alpha_j, and an elementwise phase B, U_{j+1} = z - alpha_j sigma_j U_j with
// beta_j; then the small exponential and the combine) issues 2m + 1 launches
// per step, and at 512,000 points each phase is a few microseconds of work
// behind a launch, a ramp and a grid reduction's tail.  Here the grid stays
// resident for the whole call and the phases are separated by a grid-wide
// barrier:
//   - the grid is the multi-launch path's (2 blocks of 512 threads per SM),
//     and every phase walks exactly the multi-launch kernel's work split with
//     the same arithmetic;
//   - a reduction stores the block's partial, crosses the barrier, and then
//     EVERY block adds all partials in the multi-launch last block's fixed
//     order, so every block holds the same scalars and the results equal the
//     multi-launch path's bitwise;
//   - block 0 keeps the handle's Lanczos scalars in global memory up to date
//     and forms the small exponential in its first 256 threads (a named
//     barrier) while the other blocks wait at the next grid barrier;
//   - loads of anything another block wrote during the launch go to L2
//     (ld.global.cg): an SM's L1 is not kept coherent with other SMs' stores.
// The barrier waits are bounded: a block that polls more than kGridSpins
// times sets kStatusTimeout and carries on, so the launch always ends and the
// handle reports the error at its next synchronising call.  A cooperative
// launch is refused (not queued) when the grid cannot be resident at once.
#include <cuda_runtime.h>

#include "tdse_device_common.cuh"
#include "tdse_internal.cuh"
#include "tdse_small_expm.cuh"
#include "tdse_stencil.cuh"

namespace tdse_dev {
namespace {

using namespace common;
using namespace stencil;

constexpr long long kGridSpins = 1LL << 21;   // polls of the barrier's generation (~1 us each) before giving up
constexpr int kUnrollB = 4;                   // phase B: groups loaded before use (as the B kernel)

struct PersistArgs {
  StencilIn in;              // operator; x and E are set per phase
  double2 *psi;              // U_0, rewritten by the combine
  double2 *work;             // slot 0: z; slots 1..m-1: U_j
  size_t G;
  int m;
  double dt;
  long nsteps;
  const double *etab;        // coupling at each step's mid-point
  const double *mask;
  int mask_start;
  LanczosScalars *ls;
  Reduction *red;            // the handle's (normsq after each combine)
  Reduction *rp;             // two partial buffers, used in turn
  unsigned *bar;             // barrier: arrival count, generation
  int *status;
};

// Grid-wide barrier: every block's writes before it are visible (in L2) to
// every block after it.  Once any block has given up waiting (the status
// word's timeout bit), no block waits any more, so the launch ends quickly.
__device__ __forceinline__ void grid_sync(unsigned *bar, unsigned nblocks, int *status) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = bar + 1;
    volatile int *st = status;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == nblocks - 1u) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == g) {
        if (++spins > kGridSpins || (*st & kStatusTimeout)) {
          atomicOr(status, kStatusTimeout);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// The block's partial, the barrier, then every block's fixed-order sum of all
// partials (the multi-launch last block's reduce_partials).
__device__ __forceinline__ double grid_reduce(double v, Reduction *r, double *sh, const PersistArgs &a) {
  const double b = block_sum(v, sh);
  if (threadIdx.x == 0) r->partial[blockIdx.x] = b;
  grid_sync(a.bar, gridDim.x, a.status);
  return reduce_partials(r, gridDim.x, sh);
}

// The stencil phase's work split (the multi-launch stencil kernels' walker),
// with the operand read from L2.
template <int ST, typename F>
__device__ __forceinline__ void segments_cg(const StencilIn &in, F &&f) {
  const int lane = threadIdx.x & 31;
  const int Lp1 = in.L + 1;
  const long long NJ = (in.N + 31) >> 5;
  long long s, s_end;
  warp_range(NJ * Lp1, s, s_end);
  while (s < s_end) {
    const int jg = (int)((unsigned)s / (unsigned)Lp1);
    const int l0 = (int)(s - (long long)jg * Lp1);
    const long long left = s_end - s;
    const int l1 = (left < (long long)(Lp1 - l0)) ? l0 + (int)left : Lp1;
    const int i = jg * 32 + lane;
    if (i < in.N) walk_rows<ST, 0, true, false, true>(in, i, l0, l1, f);
    s += l1 - l0;
  }
}

template <int ST>
__global__ void __launch_bounds__(kBlockJ, kStencilBlocksPerSM) lanczos_persistent_kernel(PersistArgs a) {
  __shared__ double sh[kBlockJ / 32 + 1];
  __shared__ double s_sigma[kMaxKrylov + 1], s_ratio[kMaxKrylov + 1], s_acoef[kMaxKrylov];
  __shared__ double2 s_coef[kMaxKrylov];
  __shared__ int s_k;
  const int tid = threadIdx.x, lane = tid & 31;
  const bool lead = blockIdx.x == 0;
  const size_t G = a.G;
  int par = 0;
  if (tid == 0) s_sigma[0] = __ldcg(&a.ls->sigma[0]);
  __syncthreads();
  for (long n = 0; n < a.nsteps; ++n) {
    StencilIn in = a.in;
    in.E = a.etab[n];
    for (int j = 0; j < a.m; ++j) {
      // ---- phase A (the lanczos_a kernel's arithmetic)
      const double sig = s_sigma[j];
      const double cprev = (j > 0) ? s_ratio[j] : 0.0;
      const double2 *u = (j == 0) ? a.psi : a.work + (size_t)j * G;
      const double2 *up = (j == 0) ? nullptr : ((j == 1) ? a.psi : a.work + (size_t)(j - 1) * G);
      double2 *z = a.work;
      in.x = u;
      double acc = 0.0;
      segments_cg<ST>(scaled(in, sig), [&](int, size_t idx, double2 t, double2 uu) {
        double2 o;
        if (j > 0) {
          const double2 p = __ldcg(up + idx);
          o.x = __fma_rn(-cprev, p.x, t.x);
          o.y = __fma_rn(-cprev, p.y, t.y);
        } else {
          o = t;
        }
        z[idx] = o;
        acc = __fma_rn(uu.x, o.x, acc);
        acc = __fma_rn(uu.y, o.y, acc);
      });
      const double sa = grid_reduce(acc, a.rp + par, sh, a);
      par ^= 1;
      if (tid == 0) {
        s_acoef[j] = -(sa * sig) * sig;
        if (lead) {
          a.ls->alpha[j] = sa * sig;
          a.ls->acoef[j] = -(sa * sig) * sig;
        }
      }
      __syncthreads();
      if (j + 1 >= a.m) break;
      // ---- phase B (the lanczos_b kernel's arithmetic and work split)
      const double c = s_acoef[j];
      double2 *un = a.work + (size_t)(j + 1) * G;
      double acc0 = 0.0, acc1 = 0.0;
      long long g0, g1;
      warp_range((long long)((G + 31) >> 5), g0, g1);
      for (long long gb = g0; gb < g1; gb += kUnrollB) {
        double2 zz[kUnrollB], vv[kUnrollB];
#pragma unroll
        for (int r = 0; r < kUnrollB; ++r) {
          const size_t idx = (size_t)(gb + r) * 32 + lane;
          const bool ok = (gb + r < g1) && idx < G;
          zz[r] = ok ? __ldcg(z + idx) : make_double2(0.0, 0.0);
          vv[r] = ok ? __ldcg(u + idx) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int r = 0; r < kUnrollB; ++r) {
          const size_t idx = (size_t)(gb + r) * 32 + lane;
          if ((gb + r < g1) && idx < G) {
            const double2 o = make_double2(__fma_rn(c, vv[r].x, zz[r].x), __fma_rn(c, vv[r].y, zz[r].y));
            un[idx] = o;
            acc0 = __fma_rn(o.x, o.x, acc0);
            acc1 = __fma_rn(o.y, o.y, acc1);
          }
        }
      }
      const double sb = grid_reduce(acc0 + acc1, a.rp + par, sh, a);
      par ^= 1;
      if (tid == 0) {
        const double beta = sqrt(sb);
        const double sn = (beta > 0.0) ? 1.0 / beta : 0.0;
        const double ratio = (sn > 0.0) ? s_sigma[j] * beta : 0.0;
        s_sigma[j + 1] = sn;
        s_ratio[j + 1] = ratio;
        if (lead) {
          a.ls->beta[j] = beta;
          a.ls->sigma[j + 1] = sn;
          a.ls->ratio[j + 1] = ratio;
        }
      }
      __syncthreads();
    }
    // ---- the small exponential: block 0's first kEx threads
    if (lead && tid < kEx) expm_body(a.m, a.dt, a.ls, false, ExNamedSync{});
    grid_sync(a.bar, gridDim.x, a.status);
    if (tid < kMaxKrylov) s_coef[tid] = __ldcg(&a.ls->coef[tid]);
    if (tid == 0) s_k = __ldcg(&a.ls->kdim);
    __syncthreads();
    // ---- the combine (the lanczos_combine kernel's arithmetic and work split)
    const int k = s_k;
    const int N = a.in.N;
    const double2 *U1 = a.work + G;
    double accn = 0.0;
    {
      long long g0, g1;
      warp_range((long long)((G + 31) >> 5), g0, g1);
      for (long long gi = g0; gi < g1; ++gi) {
        const size_t idx = (size_t)gi * 32 + lane;
        if (idx >= G) continue;
        const double2 u0 = __ldcg(a.psi + idx);
        double ox = __fma_rn(s_coef[0].x, u0.x, __dmul_rn(-s_coef[0].y, u0.y));
        double oy = __fma_rn(s_coef[0].x, u0.y, __dmul_rn(s_coef[0].y, u0.x));
        for (int jj = 1; jj < k; ++jj) {
          const double2 v = __ldcg(U1 + (size_t)(jj - 1) * G + idx);
          const double2 cc = s_coef[jj];
          ox = __fma_rn(cc.x, v.x, ox);
          ox = __fma_rn(-cc.y, v.y, ox);
          oy = __fma_rn(cc.x, v.y, oy);
          oy = __fma_rn(cc.y, v.x, oy);
        }
        const int jr = (int)((unsigned)idx % (unsigned)N);
        if (jr >= a.mask_start) {
          const double mv = a.mask[jr];
          ox = __dmul_rn(mv, ox);
          oy = __dmul_rn(mv, oy);
        }
        a.psi[idx] = make_double2(ox, oy);
        accn = __fma_rn(ox, ox, accn);
        accn = __fma_rn(oy, oy, accn);
      }
    }
    const double sn2 = grid_reduce(accn, a.rp + par, sh, a);
    par ^= 1;
    if (tid == 0) {
      const double nrm = sqrt(sn2);
      s_sigma[0] = (nrm > 0.0) ? 1.0 / nrm : 0.0;
      if (lead) {
        a.red->normsq = sn2;
        a.ls->psinorm = nrm;
        a.ls->sigma[0] = s_sigma[0];
        if (!isfinite(sn2)) atomicOr(a.status, kStatusNonFinite);
      }
    }
    __syncthreads();
  }
}

}  // namespace

bool lanczos_persistent_fits(int stencil) {
  int dev = 0, coop = 0, nb = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) {
    cudaGetLastError();
    return false;
  }
  const cudaError_t e = (stencil == 5)
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, lanczos_persistent_kernel<5>, kBlockJ, 0)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, lanczos_persistent_kernel<3>, kBlockJ, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return nb >= kStencilBlocksPerSM;
}

size_t lanczos_persistent_scratch_bytes() { return 2 * sizeof(Reduction) + 2 * sizeof(unsigned); }

cudaError_t launch_lanczos_persistent(const Geometry &g, const OperatorView &op, int m, double dt, long nsteps,
                                      const double *etab, double2 *psi, double2 *work, LanczosScalars *ls,
                                      Reduction *red, void *scratch, int *status, cudaStream_t st) {
  PersistArgs a;
  StencilIn &in = a.in;
  in.x = psi;
  in.diag = op.diag;
  in.rj = op.rj;
  in.kappa = op.kappa;
  in.N = g.N;
  in.L = g.L;
  in.c1 = g.c1;
  in.c2 = g.c2;
  in.E = 0.0;
  in.dscale = 1.0;
  in.rinv = nullptr;
  in.d1c = 0.0;
  a.psi = psi;
  a.work = work;
  a.G = (size_t)g.N * (g.L + 1);
  a.m = m;
  a.dt = dt;
  a.nsteps = nsteps;
  a.etab = etab;
  a.mask = op.mask;
  a.mask_start = op.mask_start;
  a.ls = ls;
  a.red = red;
  a.rp = static_cast<Reduction *>(scratch);
  a.bar = reinterpret_cast<unsigned *>(static_cast<char *>(scratch) + 2 * sizeof(Reduction));
  a.status = status;
  cudaError_t e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(g.sms * kStencilBlocksPerSM), 1, 1);
  cfg.blockDim = dim3(kBlockJ, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (g.stencil == 5) return cudaLaunchKernelEx(&cfg, lanczos_persistent_kernel<5>, a);
  return cudaLaunchKernelEx(&cfg, lanczos_persistent_kernel<3>, a);
}

}  // namespace tdse_dev
