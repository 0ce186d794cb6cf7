// Batched Lanczos propagation: many independent instances, one launch per
// Lanczos phase for the whole batch.
//
// Each instance has its own grid (N, lmax, dr, potential), pulse, absorber,
// Krylov dimension m and step dt.  Its (lmax+1) x N points are cut into
// 32-point row segments (radial-group-major, as in the single-instance
// kernels) and the segments into chunks of kChunkSegs.  A launch of phase j
// walks the chunks of every instance still active in that phase (m_i > j),
// statically split over the warps of a persistent grid.  Each chunk's partial
// sum goes to its own slot; the warp that finishes an instance's last chunk
// (per-instance arrival counter) adds that instance's chunk partials in chunk
// order.  An instance's arithmetic therefore does not depend on which other
// instances share the batch: results are bitwise the same alone and in the mix.
//
// Algorithm per instance: the Lanczos propagator of the single-instance path
// (Appendix "Lanczos methods" of arXiv 1308.1856): U_0 = psi,
// z = sigma_j H U_j - ratio_j U_{j-1}, alpha_j = sigma_j Re<U_j, z>,
// U_{j+1} = z - alpha_j sigma_j U_j, beta_j = ||U_{j+1}||, then
// c = exp(-i T dt) e_1 and psi_new = sum_j coef_j U_j, mask, ||psi_new||.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tdse_device_common.cuh"
#include "tdse_engine.h"
#include "tdse_sched.h"
#include "tdse_pulse.h"
#include "tdse_internal.cuh"
#include "tdse_stencil.cuh"

namespace tdse_dev {
namespace {

using namespace common;
using namespace stencil;

#ifndef TDSE_CHUNK_SEGS
#define TDSE_CHUNK_SEGS 64
#endif
#ifndef TDSE_CHUNK_PTS
#define TDSE_CHUNK_PTS 2048
#endif
#ifndef TDSE_TILE_ROWS
#define TDSE_TILE_ROWS 32
#endif
// Reduction chunks.  Their sizes fix each instance's summation order, so they
// are compile-time constants (the launch schedule never changes them).
constexpr int kChunkSegs = TDSE_CHUNK_SEGS;  // 32-point row segments per chunk (stencil kernels)
constexpr int kChunkPts = TDSE_CHUNK_PTS;    // consecutive points per chunk (elementwise kernels)
constexpr int kCombinePts = 2;               // points per lane whose Krylov loads the combines overlap
constexpr int kMixedCombinePts = 2;          // the same for the mixed combine, two vectors per round

__device__ __forceinline__ double field_of(const BatchDev &B, int inst) {
  return B.E[(size_t)(*B.step) * (size_t)B.cap + inst];
}

// Advance the run's step counter (one thread, after every step's last launch).
__global__ void bt_next_step(int *step) { *step += 1; }

// Index in the active list of the instance that owns global chunk gc.
__device__ __forceinline__ int find_owner(const ChunkList &cl, int gc) {
  int lo = 0, hi = cl.nact - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cl.cpre[mid] <= gc) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Add v (every lane) to the chunk's slot and, if this was the instance's last
// chunk, reduce the instance's chunk partials in order; returns true in every
// lane of the warp that must finish the instance (with the sum in `total`).
__device__ __forceinline__ bool chunk_done(const BatchDev &B, const BatchInst &I, int inst, int ci,
                                           int nchunk, double v, double &total) {
  v = warp_sum(v);
  unsigned last = 0;
  if ((threadIdx.x & 31) == 0) {
    I.partial[ci] = v;
    __threadfence();
    last = (atomicAdd(&B.ticket[inst], 1u) == (unsigned)(nchunk - 1)) ? 1u : 0u;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return false;
  __threadfence();
  double s = 0.0;
  for (int c = threadIdx.x & 31; c < nchunk; c += 32) s += __ldcg(&I.partial[c]);
  total = warp_sum(s);
  if ((threadIdx.x & 31) == 0) B.ticket[inst] = 0u;
  return true;
}

// Visit chunk ci of an instance: segments [ci*C, min((ci+1)*C, nseg)) in
// radial-group-major order; lane i of a segment owns radial index jg*32 + lane.
template <typename F>
__device__ __forceinline__ void chunk_columns(const BatchInst &I, int ci, F &&f) {
  const int lane = threadIdx.x & 31;
  const int Lp1 = I.L + 1;
  int s = ci * kChunkSegs;
  const int s_end = min(s + kChunkSegs, I.nseg);
  while (s < s_end) {
    const int jg = s / Lp1;
    const int l0 = s - jg * Lp1;
    const int l1 = min(Lp1, l0 + (s_end - s));
    const int i = jg * 32 + lane;
    if (i < I.N) f(i, l0, l1);
    s += l1 - l0;
  }
}

// The same segments as chunk_columns, for warp-collective walkers: every lane
// gets f(jg, l0, l1) (its column jg*32 + lane may be >= N).
template <typename F>
__device__ __forceinline__ void chunk_groups(const BatchInst &I, int ci, F &&f) {
  const int Lp1 = I.L + 1;
  int s = ci * kChunkSegs;
  const int s_end = min(s + kChunkSegs, I.nseg);
  while (s < s_end) {
    const int jg = s / Lp1;
    const int l0 = s - jg * Lp1;
    const int l1 = min(Lp1, l0 + (s_end - s));
    f(jg, l0, l1);
    s += l1 - l0;
  }
}

// Visit chunk ci of an instance in the elementwise layout: the kChunkPts
// consecutive points [ci*C, min((ci+1)*C, G)) of the l-major array, lane-strided
// so that every load is coalesced; f(idx, i) with i = idx mod N, the radial index.
template <typename F>
__device__ __forceinline__ void chunk_points(const BatchInst &I, int ci, F &&f) {
  const unsigned N = (unsigned)I.N;
  const unsigned G = N * (unsigned)(I.L + 1);
  const unsigned base = (unsigned)ci * kChunkPts + (threadIdx.x & 31);
  const unsigned end = min(G, (unsigned)(ci + 1) * kChunkPts);
  unsigned i = base % N;
#pragma unroll 4
  for (unsigned idx = base; idx < end; idx += 32) {
    f((size_t)idx, (int)i);
    i += 32;
    while (i >= N) i -= N;
  }
}

// As chunk_points, NQ lane-strided points at a time: the loads of all NQ
// (load(idx) -> V) are issued before the first op(idx, i, V), whose stores
// the compiler could not otherwise move loads across (the arrays may alias as
// far as it knows).  The points reach op in the same order as in chunk_points.
template <int NQ, typename Ld, typename Op>
__device__ __forceinline__ void chunk_points_xn(const BatchInst &I, int ci, Ld &&load, Op &&op) {
  const unsigned N = (unsigned)I.N;
  const unsigned G = N * (unsigned)(I.L + 1);
  const unsigned base = (unsigned)ci * kChunkPts + (threadIdx.x & 31);
  const unsigned end = min(G, (unsigned)(ci + 1) * kChunkPts);
  unsigned i = base % N;
  using V = decltype(load((size_t)0));
  for (unsigned idx = base; idx < end; idx += 32 * NQ) {
    V v[NQ];
    int iq[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      iq[q] = (int)i;
      if (idx + 32 * q < end) v[q] = load((size_t)(idx + 32 * q));
      i += 32;
      while (i >= N) i -= N;
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      if (idx + 32 * q < end) op((size_t)(idx + 32 * q), iq[q], v[q]);
  }
}
template <typename Ld, typename Op>
__device__ __forceinline__ void chunk_points_x4(const BatchInst &I, int ci, Ld &&load, Op &&op) {
  chunk_points_xn<4>(I, ci, load, op);
}

// The points of chunk_points in groups of Q consecutive lane-strided points:
// f(idx[Q], i[Q], nq) with the first nq entries valid.
template <int Q, typename F>
__device__ __forceinline__ void chunk_groups_of(const BatchInst &I, int ci, F &&f) {
  const unsigned N = (unsigned)I.N;
  const unsigned G = N * (unsigned)(I.L + 1);
  const unsigned base = (unsigned)ci * kChunkPts + (threadIdx.x & 31);
  const unsigned end = min(G, (unsigned)(ci + 1) * kChunkPts);
  unsigned i = base % N;
  for (unsigned idx = base; idx < end; idx += 32 * Q) {
    size_t ix[Q];
    int iq[Q];
    int nq = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      ix[q] = (size_t)(idx + 32 * q);
      iq[q] = (int)i;
      if (idx + 32 * q < end) nq = q + 1;
      i += 32;
      while (i >= N) i -= N;
    }
    f(ix, iq, nq);
  }
}

// Each warp takes a balanced, contiguous range of the list's chunks (warp_range).
template <typename F>
__device__ __forceinline__ void for_my_chunks(const ChunkList &cl, F &&f) {
  long long c0, c1;
  warp_range(cl.total, c0, c1);
  if (c0 >= c1) return;
  int p = find_owner(cl, (int)c0);
  for (int gc = (int)c0; gc < (int)c1; ++gc) {
    while (cl.cpre[p + 1] <= gc) ++p;
    f(cl.act[p], gc - cl.cpre[p]);
  }
}

// ---- FP64 ------------------------------------------------------------------
__device__ __forceinline__ StencilIn fp64_in(const BatchDev &B, const BatchInst &I, int inst,
                                             const double2 *x) {
  StencilIn in;
  in.x = x;
  in.diag = I.diag;
  in.rj = I.rj;
  in.kappa = I.kappa;
  in.N = I.N;
  in.L = I.L;
  in.c1 = I.c1;
  in.c2 = I.c2;
  in.E = field_of(B, inst);   // A/c for a velocity-gauge instance
  in.dscale = 1.0;
  in.rinv = I.rinv;
  in.d1c = I.d1c;
  return in;
}

// VG: the chunk list holds velocity-gauge instances only (a separate launch).
template <int ST, int PF, bool VG = false>
__global__ void __launch_bounds__(kBlockJ, kStencilBlocksPerSM)
    bt_lanczos_a_fp64(BatchDev B, ChunkList cl, int j) {
  for_my_chunks(cl, [&](int inst, int ci) {
    const BatchInst I = B.inst[inst];
    LanczosScalars *ls = B.ls + inst;
    const long long G = (long long)I.N * (I.L + 1);
    const double2 *u = (j == 0) ? I.psi : I.work + (long long)j * G;
    const double2 *up = (j <= 1) ? I.psi : I.work + (long long)(j - 1) * G;
    double2 *z = I.work;
    const double sig = ls->sigma[j];
    const double cprev = (j > 0) ? ls->ratio[j] : 0.0;
    // t = sigma_j H U_j directly (the operator scaled by sigma_j)
    const StencilIn in = scaled(fp64_in(B, I, inst, u), sig);
    double acc = 0.0;
    chunk_columns(I, ci, [&](int i, int l0, int l1) {
      walk_rows<ST, PF, true, VG>(in, i, l0, l1, [&](int, size_t idx, double2 t, double2 uc) {
        double2 o;
        if (j > 0) {
          const double2 pv = up[idx];
          o.x = __fma_rn(-cprev, pv.x, t.x);
          o.y = __fma_rn(-cprev, pv.y, t.y);
        } else {
          o = t;
        }
        z[idx] = o;
        acc = __fma_rn(uc.x, o.x, acc);
        acc = __fma_rn(uc.y, o.y, acc);
      });
    });
    double s;
    if (chunk_done(B, I, inst, ci, I.nchunk, acc, s) && (threadIdx.x & 31) == 0) {
      ls->alpha[j] = s * sig;
      ls->acoef[j] = -(s * sig) * sig;
    }
  });
}

// U_{j+1} = z - alpha_j sigma_j U_j and beta_j = ||U_{j+1}||, chunk by chunk.
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    bt_lanczos_b_fp64(BatchDev B, ChunkList cl, int j) {
  for_my_chunks(cl, [&](int inst, int ci) {
    const BatchInst I = B.inst[inst];
    LanczosScalars *ls = B.ls + inst;
    const long long G = (long long)I.N * (I.L + 1);
    const double2 *u = (j == 0) ? I.psi : I.work + (long long)j * G;
    const double2 *z = I.work;
    double2 *un = I.work + (long long)(j + 1) * G;
    const double c = ls->acoef[j];
    double acc = 0.0;
    struct ZU { double2 z, u; };
    chunk_points_x4(I, ci, [&](size_t idx) { return ZU{z[idx], u[idx]}; },
                    [&](size_t idx, int, const ZU &v) {
      const double2 o = make_double2(__fma_rn(c, v.u.x, v.z.x), __fma_rn(c, v.u.y, v.z.y));
      un[idx] = o;
      acc = __fma_rn(o.x, o.x, acc);
      acc = __fma_rn(o.y, o.y, acc);
    });
    double s;
    if (chunk_done(B, I, inst, ci, I.nchunk_e, acc, s) && (threadIdx.x & 31) == 0) {
      const double beta = sqrt(s);
      ls->beta[j] = beta;
      const double sn = (beta > 0.0) ? 1.0 / beta : 0.0;
      ls->sigma[j + 1] = sn;
      ls->ratio[j + 1] = (sn > 0.0) ? ls->sigma[j] * beta : 0.0;
    }
  });
}

// ||psi|| -> sigma_0, psinorm (FP64).
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    bt_norm_fp64(BatchDev B, ChunkList cl) {
  for_my_chunks(cl, [&](int inst, int ci) {
    const BatchInst I = B.inst[inst];
    const double2 *x = I.psi;
    double acc = 0.0;
    chunk_points_x4(I, ci, [&](size_t idx) { return x[idx]; }, [&](size_t, int, const double2 &v) {
      acc = __fma_rn(v.x, v.x, acc);
      acc = __fma_rn(v.y, v.y, acc);
    });
    double s;
    if (chunk_done(B, I, inst, ci, I.nchunk_e, acc, s) && (threadIdx.x & 31) == 0) {
      LanczosScalars *ls = B.ls + inst;
      const double nrm = sqrt(s);
      ls->psinorm = nrm;
      ls->sigma[0] = (nrm > 0.0) ? 1.0 / nrm : 0.0;
      if (!isfinite(s)) atomicOr(B.status, kStatusNonFinite);
    }
  });
}

// psi_new = sum_{j<k} coef_j U_j, mask (unless mask_on is 0: imaginary
// time), ||psi_new|| (FP64).
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    bt_combine_fp64(BatchDev B, ChunkList cl, int mask_on) {
  // the chunk's coefficients, one copy per warp
  __shared__ double2 wcoef[kElemThreads / 32][kMaxKrylov];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  for_my_chunks(cl, [&](int inst, int ci) {
    const BatchInst I = B.inst[inst];
    LanczosScalars *ls = B.ls + inst;
    const long long G = (long long)I.N * (I.L + 1);
    double2 *psi = I.psi;
    const double2 *U1 = I.work + G;
    const double *mask = I.mask;
    const int k = ls->kdim;
    __syncwarp();
    if (lane < k) wcoef[wib][lane] = ls->coef[lane];
    __syncwarp();
    const double2 c0 = wcoef[wib][0];
    double acc = 0.0;
    // kCombinePts points at a time, Krylov vector by Krylov vector
    chunk_groups_of<kCombinePts>(I, ci, [&](const size_t (&ix)[kCombinePts], const int (&iq)[kCombinePts], int nq) {
      double ox[kCombinePts], oy[kCombinePts];
#pragma unroll
      for (int q = 0; q < kCombinePts; ++q) {
        if (q < nq) {
          const double2 u0 = psi[ix[q]];
          ox[q] = __fma_rn(c0.x, u0.x, __dmul_rn(-c0.y, u0.y));
          oy[q] = __fma_rn(c0.x, u0.y, __dmul_rn(c0.y, u0.x));
        }
      }
      for (int jj = 1; jj < k; ++jj) {
        double2 u[kCombinePts];
#pragma unroll
        for (int q = 0; q < kCombinePts; ++q)
          if (q < nq) u[q] = U1[(size_t)(jj - 1) * G + ix[q]];
        const double2 c = wcoef[wib][jj];
#pragma unroll
        for (int q = 0; q < kCombinePts; ++q) {
          if (q < nq) {
            ox[q] = __fma_rn(c.x, u[q].x, ox[q]);
            ox[q] = __fma_rn(-c.y, u[q].y, ox[q]);
            oy[q] = __fma_rn(c.x, u[q].y, oy[q]);
            oy[q] = __fma_rn(c.y, u[q].x, oy[q]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kCombinePts; ++q) {
        if (q < nq) {
          if (mask_on && iq[q] >= I.mask_start) {
            const double mv = mask[iq[q]];
            ox[q] = __dmul_rn(mv, ox[q]);
            oy[q] = __dmul_rn(mv, oy[q]);
          }
          psi[ix[q]] = make_double2(ox[q], oy[q]);
          acc = __fma_rn(ox[q], ox[q], acc);
          acc = __fma_rn(oy[q], oy[q], acc);
        }
      }
    });
    double s;
    if (chunk_done(B, I, inst, ci, I.nchunk_e, acc, s) && (threadIdx.x & 31) == 0) {
      const double nrm = sqrt(s);
      ls->psinorm0 = ls->psinorm;
      ls->psinorm = nrm;
      ls->sigma[0] = (nrm > 0.0) ? 1.0 / nrm : 0.0;
      if (!isfinite(s)) atomicOr(B.status, kStatusNonFinite);
    }
  });
}

// ---- mixed precision -------------------------------------------------------
__device__ __forceinline__ MixedIn mixed_in(const BatchDev &B, const BatchInst &I, int inst,
                                            const float2 *hi, const float2 *lo, const float2 *w) {
  MixedIn in;
  in.hi = hi;
  in.lo = lo;
  in.w = w;
  in.ws = 1.f;
  in.diag = I.diagf;
  in.rj = I.rjf;
  in.kappa = I.kappaf;
  in.pf0 = nullptr;
  in.pf1 = nullptr;
  in.N = I.N;
  in.L = I.L;
  in.c1 = (float)I.c1;
  in.c2 = (float)I.c2;
  in.E = (float)field_of(B, inst);
  in.rinv = I.rinvf;   // velocity gauge only (null otherwise)
  in.d1c = (float)I.d1c;
  return in;
}

// Mixed Lanczos phase A of the velocity-gauge instances of a mixed batch (a
// launch of its own over their row-segment chunks): the register walker
// mixed_walk_rows with the (A/c) p_z coupling, in the arithmetic of the tile
// kernel (z = sigma_j H U_j - ratio_j U_{j-1} in FP32, alpha_j = sigma_j
// Re<U_j, z> from FP32 products summed in pairs, then FP64).  The operand is
// the split of psi for j = 0 and the FP32 U_j after.
template <int ST>
__global__ void __launch_bounds__(kBlockJ, kStencilBlocksPerSM)
    bt_lanczos_a_mixed_vg(BatchDev B, ChunkList cl, int j) {
  for_my_chunks(cl, [&](int inst, int ci) {
    const BatchInst I = B.inst[inst];
    LanczosScalars *ls = B.ls + inst;
    const long long G = (long long)I.N * (I.L + 1);
    const float2 *hi = I.hi, *lo = I.lo;
    float2 *z = I.mwork;
    const float2 *uprev = (j >= 2) ? I.mwork + (long long)(j - 1) * G : nullptr;
    const double sigd = ls->sigma[j];
    const float sig = (float)sigd;
    const float cprev = (j > 0) ? (float)ls->ratio[j] : 0.f;
    PairSum acc;
    auto epi = [&](int, size_t idx, float2 t, float2 u) {
      float2 o = make_float2(sig * t.x, sig * t.y);
      if (j > 0) {
        float2 up;
        if (uprev) {
          up = uprev[idx];
        } else {
          const float2 h = hi[idx], l = lo[idx];
          up = make_float2(h.x + l.x, h.y + l.y);
        }
        o.x = fmaf(-cprev, up.x, o.x);
        o.y = fmaf(-cprev, up.y, o.y);
      }
      z[idx] = o;
      acc.add(fmaf(u.x, o.x, u.y * o.y));
    };
    if (j == 0) {
      const MixedIn in = mixed_in(B, I, inst, hi, lo, nullptr);
      chunk_columns(I, ci, [&](int i, int l0, int l1) { mixed_walk_rows<ST, true, false, 0, true>(in, i, l0, l1, epi); });
    } else {
      const MixedIn in = mixed_in(B, I, inst, nullptr, nullptr, I.mwork + (long long)j * G);
      chunk_columns(I, ci, [&](int i, int l0, int l1) { mixed_walk_rows<ST, false, true, 0, true>(in, i, l0, l1, epi); });
    }
    const double accd = acc.value();
    double s;
    if (chunk_done(B, I, inst, ci, I.nchunk, accd, s) && (threadIdx.x & 31) == 0) {
      ls->alpha[j] = s * sigd;
      ls->acoef[j] = -(s * sigd) * sigd;
    }
  });
}

#include "tdse_batch_tile.cuh"

// SPLIT: U_j is U_0 = psi, read as its split (j = 0).
template <bool SPLIT>
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    bt_lanczos_b_mixed(BatchDev B, ChunkList cl, int j) {
  for_my_chunks(cl, [&](int inst, int ci) {
    const BatchInst I = B.inst[inst];
    LanczosScalars *ls = B.ls + inst;
    const long long G = (long long)I.N * (I.L + 1);
    const float2 *u = I.mwork + (long long)j * G;
    const float2 *hi = I.hi, *lo = I.lo;
    const float2 *z = I.mwork;
    float2 *un = I.mwork + (long long)(j + 1) * G;
    const float c = (float)ls->acoef[j];
    PairSum acc;
    struct ZU { float2 z, u; };
    chunk_points_x4(I, ci, [&](size_t idx) {
      float2 uu;
      if (!SPLIT) {
        uu = u[idx];
      } else {
        const float2 h = hi[idx], lw = lo[idx];
        uu = make_float2(h.x + lw.x, h.y + lw.y);
      }
      return ZU{z[idx], uu};
    }, [&](size_t idx, int, const ZU &v) {
      const float2 o = make_float2(fmaf(c, v.u.x, v.z.x), fmaf(c, v.u.y, v.z.y));
      un[idx] = o;
      acc.add(fmaf(o.x, o.x, o.y * o.y));
    });
    const double accd = acc.value();
    double s;
    if (chunk_done(B, I, inst, ci, I.nchunk_e, accd, s) && (threadIdx.x & 31) == 0) {
      const double beta = sqrt(s);
      ls->beta[j] = beta;
      const double sn = (beta > 0.0) ? 1.0 / beta : 0.0;
      ls->sigma[j + 1] = sn;
      ls->ratio[j + 1] = (sn > 0.0) ? ls->sigma[j] * beta : 0.0;
    }
  });
}

// psi -> (hi, lo) and ||psi|| (FP32 products summed in FP32 pairs, then FP64).
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    bt_split_mixed(BatchDev B, ChunkList cl) {
  for_my_chunks(cl, [&](int inst, int ci) {
    const BatchInst I = B.inst[inst];
    const double2 *x = I.psi;
    float2 *hi = I.hi, *lo = I.lo;
    PairSum acc;
    chunk_points_x4(I, ci, [&](size_t idx) { return x[idx]; }, [&](size_t idx, int, const double2 &v) {
      float2 h, lw;
      split2(v, h, lw);
      hi[idx] = h;
      lo[idx] = lw;
      acc.add(fmaf(h.x, h.x, h.y * h.y));
    });
    const double accd = acc.value();
    double s;
    if (chunk_done(B, I, inst, ci, I.nchunk_e, accd, s) && (threadIdx.x & 31) == 0) {
      LanczosScalars *ls = B.ls + inst;
      const double nrm = sqrt(s);
      ls->psinorm = nrm;
      ls->sigma[0] = (nrm > 0.0) ? 1.0 / nrm : 0.0;
      if (!isfinite(s)) atomicOr(B.status, kStatusNonFinite);
    }
  });
}

// Pair ("double-float") arithmetic in FP32: a value held as h + l with
// |l| <= ulp(h) / 2 carries about 48 bits.  Two-sum and Fast2Sum are Knuth's
// and Dekker's error-free additions; the product keeps the exact error of
// h_a h_b (an FMA) and the cross terms.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {   // |a| >= |b| or a = 0
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void pair_mul(float ah, float al, float bh, float bl, float &ph, float &pl) {
  ph = __fmul_rn(ah, bh);
  pl = __fmaf_rn(ah, bh, -ph);
  pl = __fmaf_rn(ah, bl, pl);
  pl = __fmaf_rn(al, bh, pl);
}
__device__ __forceinline__ void split1(double v, float &h, float &l) {
  h = __double2float_rn(v);
  l = __double2float_rn(v - (double)h);
}

// psi_new = coef_0 psi + sum_{j>=1} coef_j U_j, mask, ||psi_new||, with psi
// held as its split (hi + lo): the coef_0 term and the sums in pair
// arithmetic (about 48 bits), the Krylov terms in FP32 as before, and the new
// split written directly, so the step needs no FP64 instruction per point
// (an FP64 warp instruction holds its pipe 64 cycles; the FP64 form of this
// kernel was FP64-pipe bound).  The FP64 state is formed from the split when
// it is read (bt_materialize_mixed), or here too when WRITE_PSI (per-step
// observables read it after every step).
template <bool WRITE_PSI>
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    bt_combine_mixed(BatchDev B, ChunkList cl) {
  // the chunk's FP32 coefficients, converted once and kept per warp
  __shared__ float2 wcoef[kElemThreads / 32][kMaxKrylov];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  for_my_chunks(cl, [&](int inst, int ci) {
    const BatchInst I = B.inst[inst];
    LanczosScalars *ls = B.ls + inst;
    const long long G = (long long)I.N * (I.L + 1);
    double2 *psi = I.psi;
    float2 *hi = I.hi, *lo = I.lo;
    const float2 *U1 = I.mwork + G;
    const double *mask = I.mask;
    const int k = ls->kdim;
    const double2 c0 = ls->coef[0];
    float c0xh, c0xl, c0yh, c0yl;
    split1(c0.x, c0xh, c0xl);
    split1(c0.y, c0yh, c0yl);
    __syncwarp();
    if (lane < k) {
      const double2 cd = ls->coef[lane];
      wcoef[wib][lane] = make_float2((float)cd.x, (float)cd.y);
    }
    __syncwarp();
    PairSum acc;
    // kMixedCombinePts points at a time, two Krylov vectors per round (their
    // loads issued together); each point takes its terms in vector order
    constexpr int Q = kMixedCombinePts;
    chunk_groups_of<Q>(I, ci, [&](const size_t (&ix)[Q], const int (&iq)[Q], int nq) {
      float cx[Q], cy[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) cx[q] = cy[q] = 0.f;
      int jj = 1;
      for (; jj + 1 < k; jj += 2) {
        float2 u[Q], u2[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q)
          if (q < nq) {
            u[q] = U1[(size_t)(jj - 1) * G + ix[q]];
            u2[q] = U1[(size_t)jj * G + ix[q]];
          }
        const float2 c = wcoef[wib][jj], c2 = wcoef[wib][jj + 1];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          if (q < nq) {
            cx[q] = fmaf(c.x, u[q].x, cx[q]);
            cx[q] = fmaf(-c.y, u[q].y, cx[q]);
            cy[q] = fmaf(c.x, u[q].y, cy[q]);
            cy[q] = fmaf(c.y, u[q].x, cy[q]);
            cx[q] = fmaf(c2.x, u2[q].x, cx[q]);
            cx[q] = fmaf(-c2.y, u2[q].y, cx[q]);
            cy[q] = fmaf(c2.x, u2[q].y, cy[q]);
            cy[q] = fmaf(c2.y, u2[q].x, cy[q]);
          }
        }
      }
      if (jj < k) {
        float2 u[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q)
          if (q < nq) u[q] = U1[(size_t)(jj - 1) * G + ix[q]];
        const float2 c = wcoef[wib][jj];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          if (q < nq) {
            cx[q] = fmaf(c.x, u[q].x, cx[q]);
            cx[q] = fmaf(-c.y, u[q].y, cx[q]);
            cy[q] = fmaf(c.x, u[q].y, cy[q]);
            cy[q] = fmaf(c.y, u[q].x, cy[q]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        if (q < nq) {
          const float2 ph = hi[ix[q]], pl = lo[ix[q]];
          // Re: c0x px - c0y py + cx;  Im: c0x py + c0y px + cy
          float a1, a1l, a2, a2l, b1, b1l, b2, b2l;
          pair_mul(c0xh, c0xl, ph.x, pl.x, a1, a1l);
          pair_mul(c0yh, c0yl, ph.y, pl.y, a2, a2l);
          pair_mul(c0xh, c0xl, ph.y, pl.y, b1, b1l);
          pair_mul(c0yh, c0yl, ph.x, pl.x, b2, b2l);
          float sx, ex, sx2, ex2, sy, ey, sy2, ey2;
          two_sum(a1, -a2, sx, ex);
          two_sum(sx, cx[q], sx2, ex2);
          two_sum(b1, b2, sy, ey);
          two_sum(sy, cy[q], sy2, ey2);
          float oxh, oxl, oyh, oyl;
          fast_two_sum(sx2, __fadd_rn(__fadd_rn(__fsub_rn(a1l, a2l), ex), ex2), oxh, oxl);
          fast_two_sum(sy2, __fadd_rn(__fadd_rn(__fadd_rn(b1l, b2l), ey), ey2), oyh, oyl);
          if (iq[q] >= I.mask_start) {
            float mh, ml, t, tl;
            split1(mask[iq[q]], mh, ml);
            pair_mul(oxh, oxl, mh, ml, t, tl);
            fast_two_sum(t, tl, oxh, oxl);
            pair_mul(oyh, oyl, mh, ml, t, tl);
            fast_two_sum(t, tl, oyh, oyl);
          }
          hi[ix[q]] = make_float2(oxh, oyh);
          lo[ix[q]] = make_float2(oxl, oyl);
          if (WRITE_PSI) psi[ix[q]] = make_double2((double)oxh + (double)oxl, (double)oyh + (double)oyl);
          acc.add(fmaf(oxh, oxh, oyh * oyh));
        }
      }
    });
    const double accd = acc.value();
    double s;
    if (chunk_done(B, I, inst, ci, I.nchunk_e, accd, s) && (threadIdx.x & 31) == 0) {
      const double nrm = sqrt(s);
      ls->psinorm0 = ls->psinorm;
      ls->psinorm = nrm;
      ls->sigma[0] = (nrm > 0.0) ? 1.0 / nrm : 0.0;
      if (!isfinite(s)) atomicOr(B.status, kStatusNonFinite);
    }
  });
}

// The FP64 state of mixed instances first .. first + count - 1 from their
// split: psi = hi + lo (exact in FP64: the parts' mantissas do not overlap).
// A grid-stride loop per instance: no list to upload, so it queues without
// waiting for the stream.
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    bt_materialize_mixed(BatchDev B, int first, int count) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int inst = first; inst < first + count; ++inst) {
    const BatchInst I = B.inst[inst];
    const size_t G = (size_t)I.N * (I.L + 1);
    const float2 *hi = I.hi, *lo = I.lo;
    double2 *psi = I.psi;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < G; idx += stride) {
      const float2 h = hi[idx], l = lo[idx];
      psi[idx] = make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
    }
  }
}

// ---- Sec. 3: imaginary time ------------------------------------------------
// After the combine of an imaginary-time step (exp(-T dtau) in the small
// exponential, no field): psi <- psi / sqrt(dr ||psi||^2), so that the norm
// dr sum |f|^2 is one again; ||psi|| of the normalised state (the next
// step's sigma_0); and the energy estimate -ln(||psi_new|| / ||psi_old||) / dtau
// of the step (the decay rate of the norm).
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    bt_imag_normalize(BatchDev B, ChunkList cl, const double *__restrict__ dtau, double *energy) {
  for_my_chunks(cl, [&](int inst, int ci) {
    const BatchInst I = B.inst[inst];
    LanczosScalars *ls = B.ls + inst;
    const double n1 = ls->psinorm;   // every chunk reads it before the last one rewrites it
    const double sc = 1.0 / (sqrt(I.dr) * n1);
    double2 *x = I.psi;
    double acc = 0.0;
    chunk_points_x4(I, ci, [&](size_t idx) { return x[idx]; }, [&](size_t idx, int, const double2 &v) {
      const double2 o = make_double2(__dmul_rn(sc, v.x), __dmul_rn(sc, v.y));
      x[idx] = o;
      acc = __fma_rn(o.x, o.x, acc);
      acc = __fma_rn(o.y, o.y, acc);
    });
    double s;
    if (chunk_done(B, I, inst, ci, I.nchunk_e, acc, s) && (threadIdx.x & 31) == 0) {
      const double nrm = sqrt(s);
      energy[inst] = -log(n1 / ls->psinorm0) / dtau[inst];
      ls->psinorm = nrm;
      ls->sigma[0] = (nrm > 0.0) ? 1.0 / nrm : 0.0;
      if (!isfinite(s)) atomicOr(B.status, kStatusNonFinite);
    }
  });
}

// ---- Sec. 4: the dipole series ---------------------------------------------
// f_{l,i} of an instance's FP64 state, zero outside the box (the batched
// stencils have no ghost point).
__device__ __forceinline__ double2 psi_at(const BatchInst &I, int l, int i) {
  return (i >= 0 && i < I.N) ? I.psi[(size_t)l * I.N + i] : make_double2(0.0, 0.0);
}

// After a step: <z>, <zdot>, <zddot> of every instance still recording
// (Eqs. (Dipole), (DipoleVelocity), (DipoleAccel)), as the single-instance
// moments but over fixed per-instance chunks of kChunkSegs row segments.  A
// lane walks rows l0..l1-1 of its column i, carrying f_{l+1,i} to the next
// row, and accumulates (w_l = 2 kappa_{l+1} dr)
//   sn = sum_l |f_l|^2,  sre = sum_l w_l Re(f_l^* f_{l+1}),
//   sd = sum_l w_l Im(f_{l+1}^* D1raw f_l),  sc = sum_l w_l (l+1) Im(f_{l+1}^* f_l),
// then adds sn, r sre, d1c sd - sc / r and sre / r^2 to its four sums.  The
// four chunk partials go to the instance's dpart slots; the warp that
// finishes the instance's last chunk adds them in chunk order and writes
//   {t, <z>, <zdot> + (A/c) norm, -E norm - Z <1/r^2 weighted sum>}.
template <int ST>
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    bt_dipole(BatchDev B, ChunkList cl, SeriesDev S) {
  const int n = *B.step;
  const int lane = threadIdx.x & 31;
  for_my_chunks(cl, [&](int inst, int ci) {
    const long long e = S.base[inst] + n;
    if (e >= S.cap) return;   // the record is full: every chunk of the instance skips
    const BatchInst I = B.inst[inst];
    const int L = I.L;
    const double two_dr = 2.0 * I.dr;
    double q[4] = {0.0, 0.0, 0.0, 0.0};
    chunk_columns(I, ci, [&](int i, int l0, int l1) {
      double sn = 0.0, sre = 0.0, sd = 0.0, sc = 0.0;
      double2 a = psi_at(I, l0, i);
      for (int l = l0; l < l1; ++l) {
        sn = __fma_rn(a.x, a.x, __fma_rn(a.y, a.y, sn));
        if (l < L) {
          const double2 b = psi_at(I, l + 1, i);
          const double w = __dmul_rn(two_dr, I.kappa[l + 1]);
          const double w1 = __dmul_rn((double)(l + 1), w);
          const double2 p1 = psi_at(I, l, i + 1), m1 = psi_at(I, l, i - 1);
          double dx = __dsub_rn(p1.x, m1.x), dy = __dsub_rn(p1.y, m1.y);
          if (ST == 5) {
            const double2 p2 = psi_at(I, l, i + 2), m2 = psi_at(I, l, i - 2);
            dx = __dsub_rn(__fma_rn(8.0, dx, m2.x), p2.x);
            dy = __dsub_rn(__fma_rn(8.0, dy, m2.y), p2.y);
          }
          sre = __fma_rn(w, __fma_rn(a.x, b.x, __dmul_rn(a.y, b.y)), sre);
          sd = __fma_rn(w, __fma_rn(b.x, dy, -__dmul_rn(b.y, dx)), sd);
          sc = __fma_rn(w1, __fma_rn(b.x, a.y, -__dmul_rn(b.y, a.x)), sc);
          a = b;
        }
      }
      const double r = I.rj[i];
      const double rinv = 1.0 / r;
      q[0] = __dadd_rn(q[0], sn);
      q[1] = __fma_rn(r, sre, q[1]);
      q[2] = __dadd_rn(q[2], __fma_rn(I.d1c, sd, -__dmul_rn(rinv, sc)));
      q[3] = __fma_rn(__dmul_rn(rinv, rinv), sre, q[3]);
    });
    const int nd = I.nchunk_d;
    unsigned last = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = warp_sum(q[k]);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) I.dpart[(size_t)k * nd + ci] = q[k];
      __threadfence();
      last = (atomicAdd(&B.ticket[inst], 1u) == (unsigned)(nd - 1)) ? 1u : 0u;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
    double tot[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double v = 0.0;
      for (int c = lane; c < nd; c += 32) v += __ldcg(&I.dpart[(size_t)k * nd + c]);
      tot[k] = warp_sum(v);
    }
    if (lane == 0) {
      const double *tb = S.tab + 3 * ((size_t)n * S.slots + inst);
      const double norm = __dmul_rn(I.dr, tot[0]);
      double *o = S.out + 4 * ((size_t)inst * S.cap + e);
      o[0] = tb[0];
      o[1] = tot[1];
      o[2] = __fma_rn(tb[2], norm, tot[2]);
      o[3] = __fma_rn(-tb[1], norm, -__dmul_rn(I.Z, tot[3]));
      B.ticket[inst] = 0u;
    }
  });
}

// The flux through r = r_b of every listed instance (Eqs. (flux), (pad),
// (yield)), as the single-instance flux but one block row per instance: at
// the grid index ib nearest r_b (first derivative D1 as in the velocity
// gauge, zero beyond the box)
//   flux  = sum_l Im(f_l^* D1 f_l) [+ 2 (A/c) sum_l kappa_{l+1} Re(f_l^* f_{l+1})],
//   dens_k = Im(S_k^* P_k) [+ (A/c) cos(theta_k) |S_k|^2],
//   S_k = sum_l Y_l0(theta_k) f_l(r_b),  P_k = sum_l Y_l0(theta_k) (D1 f_l)(r_b),
// and the trapezoid rule advances their time integrals by (dt/2)(previous +
// current); init opens them at zero.  One warp per angle; a warp's lanes
// split the partial waves and a fixed butterfly adds their shares.  tab holds
// {t, E, A/c} per (step, slot) (init: per slot, at the current time).
constexpr int kFluxThreads = 256;

__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kFluxThreads)
    bt_flux(BatchDev B, const int *__restrict__ act, FluxDev F, const double *__restrict__ tab, int init) {
  extern __shared__ double2 fsm[];
  const int inst = act[blockIdx.y];
  const BatchInst I = B.inst[inst];
  const int L = I.L, N = I.N, ib = F.ib[inst];
  double2 *fb = fsm, *db = fsm + (L + 1);
  for (int l = threadIdx.x; l <= L; l += kFluxThreads) {
    const double2 *row = I.psi + (size_t)l * N;
    fb[l] = row[ib];
    const double2 z = make_double2(0.0, 0.0);
    const double2 p1 = ib + 1 < N ? row[ib + 1] : z, m1 = ib >= 1 ? row[ib - 1] : z;
    double dx = __dsub_rn(p1.x, m1.x), dy = __dsub_rn(p1.y, m1.y);
    if (F.stencil == 5) {
      const double2 p2 = ib + 2 < N ? row[ib + 2] : z, m2 = ib >= 2 ? row[ib - 2] : z;
      dx = __dsub_rn(__fma_rn(8.0, dx, m2.x), p2.x);
      dy = __dsub_rn(__fma_rn(8.0, dy, m2.y), p2.y);
    }
    db[l] = make_double2(__dmul_rn(dx, I.d1c), __dmul_rn(dy, I.d1c));
  }
  __syncthreads();
  const double *tb = init ? tab + 3 * (size_t)inst : tab + 3 * ((size_t)(*B.step) * F.slots + inst);
  const double ac = tb[2];
  const double half_dt = init ? 0.0 : 0.5 * F.dt[inst];
  double *st = F.state + (size_t)inst * (2 + 2 * (size_t)F.nt);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (blockIdx.x == 0 && warp == 0) {
    double tot = 0.0;
    for (int l = lane; l <= L; l += 32) {
      tot = __fma_rn(fb[l].x, db[l].y, __fma_rn(-fb[l].y, db[l].x, tot));
      if (ac != 0.0 && l < L)
        tot = __fma_rn(2.0 * ac * I.kappa[l + 1], __fma_rn(fb[l].x, fb[l + 1].x, __dmul_rn(fb[l].y, fb[l + 1].y)),
                       tot);
    }
    tot = warp_allsum(tot);
    if (lane == 0) {
      st[1] = init ? 0.0 : __fma_rn(half_dt, __dadd_rn(st[0], tot), st[1]);
      st[0] = tot;
    }
  }
  const int k = blockIdx.x * (kFluxThreads / 32) + warp;
  if (k >= F.nt) return;
  const double *yk = F.y + (size_t)k * F.ystride;
  double sx = 0.0, sy = 0.0, px = 0.0, py = 0.0;
  for (int l = lane; l <= L; l += 32) {
    const double y = yk[l];
    sx = __fma_rn(y, fb[l].x, sx);
    sy = __fma_rn(y, fb[l].y, sy);
    px = __fma_rn(y, db[l].x, px);
    py = __fma_rn(y, db[l].y, py);
  }
  sx = warp_allsum(sx);
  sy = warp_allsum(sy);
  px = warp_allsum(px);
  py = warp_allsum(py);
  if (lane == 0) {
    double dens = __fma_rn(sx, py, -__dmul_rn(sy, px));
    if (ac != 0.0) dens = __fma_rn(ac * F.ct[k], __fma_rn(sx, sx, __dmul_rn(sy, sy)), dens);
    double *now = st + 2, *acc = st + 2 + F.nt;
    acc[k] = init ? 0.0 : __fma_rn(half_dt, __dadd_rn(now[k], dens), acc[k]);
    now[k] = dens;
  }
}

}  // namespace
}  // namespace tdse_dev


// ===========================================================================
// Host side: the engine
// ===========================================================================
namespace tdse_dev {
namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct Layout {
  size_t psi, diag, diagf, hi, lo, work, mwork, rj, mask, kappa, rjf, kappaf, partial, dpart, ref0, rinv, rinvf,
      total;
};

// Tiles of the mixed tile kernel on an N x (L+1) grid.
int tile_count(int N, int L) { return ((N + kTileCols - 1) / kTileCols) * ((L + kTileRows) / kTileRows); }

Layout layout_of(const tdse_instance_spec &s, int precision) {
  const size_t N = (size_t)s.N, Lp1 = (size_t)s.lmax + 1, G = N * Lp1, m = (size_t)s.krylov;
  const size_t nseg = ((N + 31) / 32) * Lp1;
  const size_t nchunk = std::max({(nseg + kChunkSegs - 1) / kChunkSegs, (G + kChunkPts - 1) / kChunkPts,
                                  (size_t)tile_count(s.N, s.lmax)});
  const bool mixed = precision == TDSE_MIXED;
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += align_up(bytes);
    return at;
  };
  const size_t none = ~(size_t)0;
  L.psi = take(16 * G);
  L.diag = mixed ? none : take(8 * G);
  L.work = mixed ? none : take(16 * G * m);
  L.diagf = mixed ? take(4 * G) : none;
  L.hi = mixed ? take(8 * G) : none;
  L.lo = mixed ? take(8 * G) : none;
  L.mwork = mixed ? take(8 * G * m) : none;
  L.rj = take(8 * N);
  L.mask = take(8 * N);
  L.kappa = take(8 * (Lp1 + 1));
  L.rjf = mixed ? take(4 * N) : none;
  L.kappaf = mixed ? take(4 * (Lp1 + 1)) : none;
  L.partial = take(8 * nchunk);
  L.dpart = take(8 * 4 * ((nseg + kChunkSegs - 1) / kChunkSegs));
  L.ref0 = take(16 * N);
  L.rinv = (!mixed && s.gauge == TDSE_GAUGE_VELOCITY) ? take(8 * N) : none;
  L.rinvf = (mixed && s.gauge == TDSE_GAUGE_VELOCITY) ? take(4 * N) : none;
  L.total = off;
  return L;
}

// The coupling's time factor of an instance at t: E(t), or A(t)/c in the velocity gauge.
double pulse_at(const tdse_instance_spec &s, double t) {
  const PulseParams p{s.E0, s.omega, s.ncycles, s.cep, s.pulse_shape};
  return s.gauge == TDSE_GAUGE_VELOCITY ? pulse_vecpot(p, t) / kLightAU : pulse_field(p, t);
}

ChunkList list_at(const int *base, int off, int nact, int total) {
  ChunkList cl;
  cl.act = base + off;
  cl.cpre = base + off + nact;
  cl.nact = nact;
  cl.total = total;
  return cl;
}

}  // namespace

#define EN_CUDA(call, what)                                                             \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(TDSE_ERR_CUDA, std::string(what) + ": " +        \
                                                         cudaGetErrorString(e_));       \
  } while (0)

bool valid_spec(const tdse_instance_spec &s) {
  if (s.N < 1 || s.lmax < 0 || !(s.dr > 0.0) || !(s.dt > 0.0) || !std::isfinite(s.dt) ||
      !std::isfinite(s.dr) || !std::isfinite(s.Z))
    return false;
  if (s.krylov < 1 || s.krylov > TDSE_MAX_KRYLOV) return false;
  if (!std::isfinite(s.E0) || !std::isfinite(s.omega) || !std::isfinite(s.ncycles) ||
      !std::isfinite(s.cep) || !std::isfinite(s.absorber_r) || !std::isfinite(s.r_b))
    return false;
  if (s.E0 != 0.0 && (!(s.omega > 0.0) || !(s.ncycles > 0.0))) return false;
  if ((s.gauge != TDSE_GAUGE_LENGTH && s.gauge != TDSE_GAUGE_VELOCITY) ||
      (s.pulse_shape != TDSE_PULSE_SIN2_E && s.pulse_shape != TDSE_PULSE_SIN2_A))
    return false;
  // segment and chunk indices are 32-bit in the kernels
  const long long nseg = (long long)((s.N + 31) / 32) * (s.lmax + 1);
  if (nseg > (1LL << 30) || (long long)s.N * (s.lmax + 1) >= (1LL << 31)) return false;
  return true;
}

size_t instance_bytes(const tdse_instance_spec &s, int precision) {
  return layout_of(s, precision).total;
}

Engine::~Engine() {
  if (stream) cudaStreamSynchronize(stream);
  for (CachedGraph &g : graphs) cudaGraphExecDestroy(g.exec);
  cudaFree(inst);
  cudaFree(ls);
  cudaFree(ticket);
  cudaFree(status);
  cudaFree(m_dev);
  cudaFree(dt_dev);
  cudaFree(E_dev);
  cudaFree(step_dev);
  cudaFree(lists);
  cudaFree(obs_partials);   // obs_out points into this block
  cudaFree(obs_ticket);
  cudaFree(ser);
  cudaFree(ser_base);
  cudaFree(ser_tab);
  cudaFree(flux_state);
  cudaFree(flux_y);
  cudaFree(flux_ct);
  cudaFree(flux_ib);
  cudaFree(flux_slots);
  cudaFree(imag_e);
  for (auto &mk : marks) {
    cudaEventDestroy(mk.a);
    cudaEventDestroy(mk.b);
  }
  if (own_stream) cudaStreamDestroy(own_stream);
}

int Engine::fail(int code, const std::string &msg) {
  err = msg;
  if (code == TDSE_ERR_CUDA) poisoned = true;
  return code;
}

int Engine::init(int cap, int st, int prec) {
  capacity = cap;
  stencil = st;
  precision = prec;
  int dev = 0;
  EN_CUDA(cudaGetDevice(&dev), "device");
  EN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attributes");
  EN_CUDA(cudaStreamCreateWithFlags(&own_stream, cudaStreamNonBlocking), "stream");
  stream = own_stream;
  hinst.assign(cap, BatchInst{});
  spec.assign(cap, tdse_instance_spec{});
  nstep.assign(cap, 0);
  tstart.assign(cap, 0.0);
  placed.assign(cap, 0);
  norm_valid.assign(cap, 0);
  ser_count.assign(cap, 0);
  psi_stale.assign(cap, 0);
  const bool ok = cudaMalloc(&inst, sizeof(BatchInst) * cap) == cudaSuccess &&
                  cudaMalloc(&ls, sizeof(LanczosScalars) * cap) == cudaSuccess &&
                  cudaMalloc(&ticket, sizeof(unsigned) * cap) == cudaSuccess &&
                  cudaMalloc(&status, sizeof(int)) == cudaSuccess &&
                  cudaMalloc(&m_dev, sizeof(int) * cap) == cudaSuccess &&
                  cudaMalloc(&dt_dev, sizeof(double) * cap) == cudaSuccess &&
                  cudaMalloc(&obs_ticket, sizeof(unsigned)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return fail(TDSE_ERR_OOM, "engine descriptors");
  }
  EN_CUDA(cudaMemsetAsync(ls, 0, sizeof(LanczosScalars) * cap, stream), "clear");
  EN_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned) * cap, stream), "clear");
  EN_CUDA(cudaMemsetAsync(status, 0, sizeof(int), stream), "clear");
  EN_CUDA(cudaMemsetAsync(m_dev, 0, sizeof(int) * cap, stream), "clear");
  EN_CUDA(cudaMemsetAsync(dt_dev, 0, sizeof(double) * cap, stream), "clear");
  EN_CUDA(cudaMemsetAsync(obs_ticket, 0, sizeof(unsigned), stream), "clear");
  EN_CUDA(cudaStreamSynchronize(stream), "sync");
  return TDSE_OK;
}

int Engine::ensure(void **p, size_t &cap, size_t bytes, const char *what) {
  if (bytes <= cap) return TDSE_OK;
  EN_CUDA(cudaStreamSynchronize(stream), "sync before growing a buffer");
  cudaFree(*p);
  *p = nullptr;
  cap = 0;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(TDSE_ERR_OOM, what);
  }
  cap = bytes;
  return TDSE_OK;
}

int Engine::place(int slot, const tdse_instance_spec &s, void *mem) {
  if (poisoned) return TDSE_ERR_STATE;
  if (slot < 0 || slot >= capacity || !mem || ((uintptr_t)mem & (kAlign - 1)))
    return fail(TDSE_ERR_ARG, "bad slot or unaligned instance memory");
  if (!valid_spec(s)) return fail(TDSE_ERR_ARG, "invalid instance spec");
  const bool mixed = precision == TDSE_MIXED;
  const Layout Lo = layout_of(s, precision);
  char *base = static_cast<char *>(mem);
  const int N = s.N, L = s.lmax;
  const size_t G = (size_t)N * (L + 1);
  BatchInst I{};
  I.N = N;
  I.L = L;
  I.m = s.krylov;
  I.nseg = (int)((size_t)((N + 31) / 32) * (L + 1));
  // reduction chunks of the stencil kernel: 64 row segments (FP64 and the
  // mixed velocity gauge), or tiles of 256 columns x kTileRows rows (the
  // mixed tile kernel)
  const bool vg = s.gauge == TDSE_GAUGE_VELOCITY;
  I.nchunk = (mixed && !vg) ? tile_count(N, L) : (I.nseg + kChunkSegs - 1) / kChunkSegs;
  I.nchunk_e = (int)((G + kChunkPts - 1) / kChunkPts);
  I.nchunk_d = (I.nseg + kChunkSegs - 1) / kChunkSegs;
  I.dr = s.dr;
  I.Z = s.Z;
  const double h2 = s.dr * s.dr;
  double c0;
  if (stencil == 5) {
    c0 = 30.0 / (24.0 * h2);
    I.c1 = -16.0 / (24.0 * h2);
    I.c2 = 1.0 / (24.0 * h2);
  } else {
    c0 = 1.0 / h2;
    I.c1 = -0.5 / h2;
    I.c2 = 0.0;
  }
  I.psi = reinterpret_cast<double2 *>(base + Lo.psi);
  I.rj = reinterpret_cast<double *>(base + Lo.rj);
  I.mask = reinterpret_cast<double *>(base + Lo.mask);
  I.kappa = reinterpret_cast<double *>(base + Lo.kappa);
  I.partial = reinterpret_cast<double *>(base + Lo.partial);
  I.dpart = reinterpret_cast<double *>(base + Lo.dpart);
  I.ref0 = reinterpret_cast<double2 *>(base + Lo.ref0);
  I.gauge = s.gauge;
  I.d1c = (stencil == 5) ? 1.0 / (12.0 * s.dr) : 1.0 / (2.0 * s.dr);
  I.rinv = (!mixed && vg) ? reinterpret_cast<double *>(base + Lo.rinv) : nullptr;
  I.rinvf = (mixed && vg) ? reinterpret_cast<float *>(base + Lo.rinvf) : nullptr;
  if (mixed) {
    I.diagf = reinterpret_cast<float *>(base + Lo.diagf);
    I.hi = reinterpret_cast<float2 *>(base + Lo.hi);
    I.lo = reinterpret_cast<float2 *>(base + Lo.lo);
    I.mwork = reinterpret_cast<float2 *>(base + Lo.mwork);
    I.rjf = reinterpret_cast<float *>(base + Lo.rjf);
    I.kappaf = reinterpret_cast<float *>(base + Lo.kappaf);
  } else {
    I.diag = reinterpret_cast<double *>(base + Lo.diag);
    I.work = reinterpret_cast<double2 *>(base + Lo.work);
  }
  // tables (host), r_j = j dr, j = 1..N
  std::vector<double> rj(N), kap(L + 2), msk(N, 1.0);
  for (int j = 0; j < N; ++j) rj[j] = (double)(j + 1) * s.dr;
  kap[0] = 0.0;
  for (int l = 1; l <= L; ++l) {
    const double ll = (double)l * (double)l;
    kap[l] = std::sqrt(ll / (4.0 * ll - 1.0));
  }
  kap[L + 1] = 0.0;
  I.mask_start = N;
  const double R = rj[N - 1], ra = s.absorber_r;
  if (ra < R) {
    for (int j = 0; j < N; ++j) {
      const double r = rj[j];
      if (r > ra) {
        if (I.mask_start == N) I.mask_start = j;
        msk[j] = std::pow(std::cos(0.5 * M_PI * (r - ra) / (R - ra)), 0.125);
      }
    }
  }
  // normalised 1s state in l = 0 (also the p_ground reference)
  std::vector<double> ref(2 * (size_t)N, 0.0);
  double nrm = 0.0;
  for (int j = 0; j < N; ++j) {
    const double p = 2.0 * rj[j] * std::exp(-rj[j]);
    ref[2 * j] = p;
    nrm += p * p;
  }
  const double sc = 1.0 / std::sqrt(s.dr * nrm);
  for (int j = 0; j < N; ++j) ref[2 * j] *= sc;
  cudaStream_t st = stream;
  EN_CUDA(cudaMemsetAsync(I.psi, 0, sizeof(double2) * G, st), "clear state");
  EN_CUDA(cudaMemcpyAsync(I.psi, ref.data(), sizeof(double) * ref.size(), cudaMemcpyHostToDevice, st), "state");
  EN_CUDA(cudaMemcpyAsync(I.ref0, ref.data(), sizeof(double) * ref.size(), cudaMemcpyHostToDevice, st), "reference");
  EN_CUDA(cudaMemcpyAsync((void *)I.rj, rj.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st), "r table");
  EN_CUDA(cudaMemcpyAsync((void *)I.mask, msk.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st), "mask");
  EN_CUDA(cudaMemcpyAsync((void *)I.kappa, kap.data(), sizeof(double) * (L + 2), cudaMemcpyHostToDevice, st), "kappa");
  std::vector<double> ri;
  if (I.rinv) {
    ri.resize(N);
    for (int j = 0; j < N; ++j) ri[j] = 1.0 / rj[j];
    EN_CUDA(cudaMemcpyAsync((void *)I.rinv, ri.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st), "1/r table");
  }
  if (mixed) {
    std::vector<float> df(G), rf(N), kf(L + 2);
    for (int l = 0; l <= L; ++l) {
      const double cent = 0.5 * (double)l * (double)(l + 1);
      for (int j = 0; j < N; ++j) {
        const double r = rj[j];
        df[(size_t)l * N + j] = (float)((c0 + cent / (r * r) - s.Z / r) - c0);
      }
    }
    for (int j = 0; j < N; ++j) rf[j] = (float)rj[j];
    if (I.rinvf) {
      std::vector<float> rif(N);
      for (int j = 0; j < N; ++j) rif[j] = (float)(1.0 / rj[j]);
      EN_CUDA(cudaMemcpyAsync((void *)I.rinvf, rif.data(), sizeof(float) * N, cudaMemcpyHostToDevice, st),
              "1/r table");
      EN_CUDA(cudaStreamSynchronize(st), "sync 1/r table");
    }
    for (int l = 0; l < L + 2; ++l) kf[l] = (float)kap[l];
    EN_CUDA(cudaMemcpyAsync((void *)I.diagf, df.data(), sizeof(float) * G, cudaMemcpyHostToDevice, st), "diag");
    EN_CUDA(cudaMemcpyAsync((void *)I.rjf, rf.data(), sizeof(float) * N, cudaMemcpyHostToDevice, st), "r table");
    EN_CUDA(cudaMemcpyAsync((void *)I.kappaf, kf.data(), sizeof(float) * (L + 2), cudaMemcpyHostToDevice, st), "kappa");
    EN_CUDA(cudaStreamSynchronize(st), "sync tables");
  } else {
    std::vector<double> diag(G);
    for (int l = 0; l <= L; ++l) {
      const double cent = 0.5 * (double)l * (double)(l + 1);
      for (int j = 0; j < N; ++j) {
        const double r = rj[j];
        diag[(size_t)l * N + j] = c0 + cent / (r * r) - s.Z / r;
      }
    }
    EN_CUDA(cudaMemcpyAsync((void *)I.diag, diag.data(), sizeof(double) * G, cudaMemcpyHostToDevice, st), "diag");
    EN_CUDA(cudaStreamSynchronize(st), "sync tables");
  }
  const int m = s.krylov;
  const double dt = s.dt;
  EN_CUDA(cudaMemcpyAsync(inst + slot, &I, sizeof(BatchInst), cudaMemcpyHostToDevice, st), "descriptor");
  EN_CUDA(cudaMemcpyAsync(m_dev + slot, &m, sizeof(int), cudaMemcpyHostToDevice, st), "descriptor");
  EN_CUDA(cudaMemcpyAsync(dt_dev + slot, &dt, sizeof(double), cudaMemcpyHostToDevice, st), "descriptor");
  EN_CUDA(cudaStreamSynchronize(st), "sync descriptor");
  hinst[slot] = I;
  spec[slot] = s;
  nstep[slot] = 0;
  tstart[slot] = 0.0;
  placed[slot] = 1;
  norm_valid[slot] = 0;
  ser_count[slot] = 0;
  psi_stale[slot] = 0;
  return TDSE_OK;
}

void Engine::clear(int slot) {
  if (slot < 0 || slot >= capacity) return;
  placed[slot] = 0;
  norm_valid[slot] = 0;
  hinst[slot] = BatchInst{};
}

double Engine::time_of(int slot) const {
  return (slot >= 0 && slot < capacity) ? tstart[slot] + (double)nstep[slot] * spec[slot].dt : 0.0;
}

int Engine::set_time(int slot, double t) {
  if (poisoned) return TDSE_ERR_STATE;
  if (slot < 0 || slot >= capacity || !placed[slot] || !std::isfinite(t))
    return fail(TDSE_ERR_ARG, "bad instance or non-finite time");
  tstart[slot] = t;
  nstep[slot] = 0;
  return TDSE_OK;
}

long long Engine::steps_of(int slot) const { return (slot >= 0 && slot < capacity) ? nstep[slot] : 0; }

cudaEvent_t Engine::prof_begin(int kind) {
  if (!profiling) return nullptr;
  if (nmarks == marks.size()) {
    Mark mk;
    if (cudaEventCreate(&mk.a) != cudaSuccess || cudaEventCreate(&mk.b) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    marks.push_back(mk);
  }
  Mark &mk = marks[nmarks++];
  mk.kind = kind;
  cudaEventRecord(mk.a, stream);
  return mk.b;
}

void Engine::prof_end(cudaEvent_t e) {
  if (e) cudaEventRecord(e, stream);
}

int Engine::prof_collect() {
  EN_CUDA(cudaStreamSynchronize(stream), "sync profile");
  for (size_t i = 0; i < nmarks; ++i) {
    float ms = 0.f;
    EN_CUDA(cudaEventElapsedTime(&ms, marks[i].a, marks[i].b), "event time");
    prof_ms[marks[i].kind] += ms;
    prof_n[marks[i].kind] += 1;
  }
  nmarks = 0;
  return TDSE_OK;
}

int Engine::profile(int enable) {
  if (poisoned) return TDSE_ERR_STATE;
  if (profiling) {
    const int rc = prof_collect();
    if (rc) return rc;
  }
  if (enable)
    for (int k = 0; k < TDSE_K_COUNT; ++k) {
      prof_ms[k] = 0.0;
      prof_n[k] = 0;
    }
  profiling = enable != 0;
  return TDSE_OK;
}

int Engine::profile_read(int kind, double *total_ms, long long *n) {
  if (poisoned) return TDSE_ERR_STATE;
  if (kind < 0 || kind >= TDSE_K_COUNT) return fail(TDSE_ERR_ARG, "unknown kernel kind");
  if (profiling) {
    const int rc = prof_collect();
    if (rc) return rc;
  }
  if (total_ms) *total_ms = prof_ms[kind];
  if (n) *n = prof_n[kind];
  return TDSE_OK;
}

int Engine::sync() {
  if (poisoned) return TDSE_ERR_STATE;
  EN_CUDA(cudaStreamSynchronize(stream), "sync");
  return check_status();
}

// A wait of the mixed tile kernel that gave up (kStatusTimeout): the results
// of that launch are not trustworthy, so the engine is poisoned.
int Engine::check_status() {
  int st = 0;
  EN_CUDA(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, stream), "read status");
  EN_CUDA(cudaStreamSynchronize(stream), "sync status");
  if (st & kStatusTimeout) {
    poisoned = true;
    return fail(TDSE_ERR_CUDA, "a staged copy of the mixed stencil kernel did not arrive in time");
  }
  return TDSE_OK;
}

int Engine::set_stream(void *cuda_stream) {
  if (poisoned) return TDSE_ERR_STATE;
  EN_CUDA(cudaStreamSynchronize(stream), "sync");
  stream = cuda_stream ? (cudaStream_t)cuda_stream : own_stream;
  return TDSE_OK;
}

int Engine::set_state(int slot, const double *F) {
  if (poisoned) return TDSE_ERR_STATE;
  if (slot < 0 || slot >= capacity || !placed[slot] || !F) return fail(TDSE_ERR_ARG, "bad instance or null state");
  const BatchInst &I = hinst[slot];
  const size_t G = (size_t)I.N * (I.L + 1);
  EN_CUDA(cudaMemcpyAsync(I.psi, F, sizeof(double2) * G, cudaMemcpyHostToDevice, stream), "set state");
  EN_CUDA(cudaStreamSynchronize(stream), "sync");
  norm_valid[slot] = 0;
  psi_stale[slot] = 0;
  return TDSE_OK;
}

int Engine::get_state(int slot, double *F) {
  if (poisoned) return TDSE_ERR_STATE;
  if (slot < 0 || slot >= capacity || !placed[slot] || !F) return fail(TDSE_ERR_ARG, "bad instance or null state");
  int rc = materialize({slot});
  if (rc) return rc;
  const BatchInst &I = hinst[slot];
  const size_t G = (size_t)I.N * (I.L + 1);
  EN_CUDA(cudaMemcpyAsync(F, I.psi, sizeof(double2) * G, cudaMemcpyDeviceToHost, stream), "get state");
  EN_CUDA(cudaStreamSynchronize(stream), "sync");
  return TDSE_OK;
}

int Engine::copy_states(const std::vector<int> &slots, double *F, bool to_device) {
  if (poisoned) return TDSE_ERR_STATE;
  if (!F) return fail(TDSE_ERR_ARG, "null state buffer");
  for (int slot : slots)
    if (slot < 0 || slot >= capacity || !placed[slot]) return fail(TDSE_ERR_ARG, "bad instance");
  if (!to_device) {
    const int rc = materialize(slots);
    if (rc) return rc;
  }
  size_t off = 0;
  for (int slot : slots) {
    if (slot < 0 || slot >= capacity || !placed[slot]) return fail(TDSE_ERR_ARG, "bad instance");
    const BatchInst &I = hinst[slot];
    const size_t G = (size_t)I.N * (I.L + 1);
    if (to_device) {
      EN_CUDA(cudaMemcpyAsync(I.psi, F + off, sizeof(double2) * G, cudaMemcpyHostToDevice, stream), "set states");
      norm_valid[slot] = 0;
      psi_stale[slot] = 0;
    } else {
      EN_CUDA(cudaMemcpyAsync(F + off, I.psi, sizeof(double2) * G, cudaMemcpyDeviceToHost, stream), "get states");
    }
    off += 2 * G;
  }
  EN_CUDA(cudaStreamSynchronize(stream), "sync states");
  return TDSE_OK;
}

int Engine::materialize(const std::vector<int> &slots) {
  if (poisoned) return TDSE_ERR_STATE;
  if (precision != TDSE_MIXED) return TDSE_OK;
  std::vector<int> ids;
  for (int s : slots)
    if (s >= 0 && s < capacity && placed[s] && psi_stale[s]) ids.push_back(s);
  if (ids.empty()) return TDSE_OK;
  std::sort(ids.begin(), ids.end());
  ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
  const BatchDev B = device_view();
  const unsigned grid = (unsigned)(sms * sched.eblocks);
  // one launch per run of consecutive slots
  for (size_t q = 0; q < ids.size();) {
    size_t r = q + 1;
    while (r < ids.size() && ids[r] == ids[r - 1] + 1) ++r;
    bt_materialize_mixed<<<grid, kElemThreads, 0, stream>>>(B, ids[q], (int)(r - q));
    ++launches;
    EN_CUDA(cudaGetLastError(), "materialize");
    q = r;
  }
  for (int id : ids) psi_stale[id] = 0;
  return TDSE_OK;
}

// Append the chunk list of `ids` (stencil, elementwise or dipole chunks) to the host
// staging; list_off receives its offset, the return value its chunk count.
int Engine::launch_lists(const std::vector<int> &ids, ListKind kind, int &list_off) {
  list_off = (int)hlists.size();
  hlists.insert(hlists.end(), ids.begin(), ids.end());
  int tot = 0;
  hlists.push_back(0);
  for (int id : ids) {
    const BatchInst &I = hinst[id];
    tot += kind == kListElem ? I.nchunk_e : kind == kListRows ? I.nchunk_d : I.nchunk;
    hlists.push_back(tot);
  }
  return tot;
}

namespace {

constexpr long kGraphMinSteps = 3;   // segments this long replay one captured step graph
constexpr size_t kGraphCache = 8;    // captured step graphs kept across runs

template <int ST, int PF>
void launch_a_pf(unsigned grid, cudaStream_t st, const BatchDev &B, const ChunkList &cl, int j) {
  bt_lanczos_a_fp64<ST, PF><<<grid, kBlockJ, 0, st>>>(B, cl, j);
}

// The mixed tile kernel: dynamic shared memory of its ring of D row slots,
// raised above the 48 KB default once per instantiation.
template <int ST, int D, int MODE>
cudaError_t launch_tile_mode(unsigned grid, cudaStream_t st, const BatchDev &B, const ChunkList &cl, int j) {
  constexpr int bytes = tile_smem_bytes<MODE, D>();
  static bool configured = false;
  if (!configured) {
    const cudaError_t e = cudaFuncSetAttribute(bt_lanczos_a_mixed_tile<ST, MODE, D>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  bt_lanczos_a_mixed_tile<ST, MODE, D><<<grid, kTileBlock, bytes, st>>>(B, cl, j);
  return cudaGetLastError();
}

template <int ST, int D>
cudaError_t launch_tile(unsigned grid, cudaStream_t st, const BatchDev &B, const ChunkList &cl, int j) {
  if (j == 0) return launch_tile_mode<ST, D, 0>(grid, st, B, cl, j);
  if (j == 1) return launch_tile_mode<ST, D, 1>(grid, st, B, cl, j);
  return launch_tile_mode<ST, D, 2>(grid, st, B, cl, j);
}

// ring of row slots (schedule ring_rows 0, 3, 5 -> 4, 8, 12 slots: 1, 5 or 9
// rows in flight beyond the three the stencil holds)
template <int ST>
cudaError_t launch_tile_ring(int ring, unsigned grid, cudaStream_t st, const BatchDev &B, const ChunkList &cl,
                             int j) {
  if (ring == 0) return launch_tile<ST, 4>(grid, st, B, cl, j);
  if (ring == 3) return launch_tile<ST, 8>(grid, st, B, cl, j);
  return launch_tile<ST, 12>(grid, st, B, cl, j);
}

template <int ST>
void launch_a_st(int pf, unsigned grid, cudaStream_t st, const BatchDev &B, const ChunkList &cl, int j) {
  switch (pf) {
    case 0: launch_a_pf<ST, 0>(grid, st, B, cl, j); break;
    case 3: launch_a_pf<ST, 3>(grid, st, B, cl, j); break;
    case 10: launch_a_pf<ST, 10>(grid, st, B, cl, j); break;
    default: launch_a_pf<ST, 6>(grid, st, B, cl, j); break;
  }
}

template <int ST>
void launch_a_vg_st(int pf, unsigned grid, cudaStream_t st, const BatchDev &B, const ChunkList &cl, int j) {
  switch (pf) {
    case 0: bt_lanczos_a_fp64<ST, 0, true><<<grid, kBlockJ, 0, st>>>(B, cl, j); break;
    case 3: bt_lanczos_a_fp64<ST, 3, true><<<grid, kBlockJ, 0, st>>>(B, cl, j); break;
    case 10: bt_lanczos_a_fp64<ST, 10, true><<<grid, kBlockJ, 0, st>>>(B, cl, j); break;
    default: bt_lanczos_a_fp64<ST, 6, true><<<grid, kBlockJ, 0, st>>>(B, cl, j); break;
  }
}

}  // namespace

void Engine::drop_graphs() {
  last_eager.clear();
  if (graphs.empty()) return;
  cudaStreamSynchronize(stream);
  for (CachedGraph &g : graphs) cudaGraphExecDestroy(g.exec);
  graphs.clear();
}

// Everything a captured step of this segment depends on: the schedule, the
// device buffers its launches point into, the segment's list offsets and
// counts and the chunk lists themselves (the instance descriptors, Krylov
// dimensions and steps are read on the device when the graph runs).
std::vector<long long> Engine::segment_key(const Segment &sg) const {
  std::vector<long long> k;
  k.reserve(32 + 9 * sg.off.size() + hlists.size());
  k.push_back(precision);
  k.push_back(stencil);
  k.push_back(sched.pf);
  k.push_back(sched.ring);
  k.push_back(sched.sblocks);
  k.push_back(sched.eblocks);
  k.push_back(capacity);
  k.push_back(sg.maxm);
  for (const void *p : {(const void *)inst, (const void *)ls, (const void *)ticket, (const void *)status,
                        (const void *)m_dev, (const void *)dt_dev, (const void *)E_dev, (const void *)step_dev,
                        (const void *)lists, (const void *)ser, (const void *)ser_base, (const void *)ser_tab})
    k.push_back((long long)(uintptr_t)p);
  for (const void *p : {(const void *)flux_state, (const void *)flux_y, (const void *)flux_ct,
                        (const void *)flux_ib})
    k.push_back((long long)(uintptr_t)p);
  k.push_back(flux_nt);
  k.push_back(run_imag ? 1 : 0);
  k.push_back((long long)(uintptr_t)imag_e);
  k.push_back(ser_cap);
  k.push_back(sg.doff);
  k.push_back(sg.dnact);
  k.push_back(sg.dtotal);
  for (const std::vector<int> *v : {&sg.off, &sg.nact, &sg.total, &sg.voff, &sg.vnact, &sg.vtotal, &sg.eoff,
                                    &sg.enact, &sg.etotal}) {
    k.push_back((long long)v->size());
    k.insert(k.end(), v->begin(), v->end());
  }
  k.push_back((long long)hlists.size());
  k.insert(k.end(), hlists.begin(), hlists.end());
  return k;
}

SeriesDev Engine::series_view() const {
  SeriesDev S;
  S.out = ser;
  S.cap = ser_cap;
  S.base = ser_base;
  S.tab = ser_tab;
  S.slots = capacity;
  return S;
}

FluxDev Engine::flux_view() const {
  FluxDev F;
  F.state = flux_state;
  F.y = flux_y;
  F.ct = flux_ct;
  F.ib = flux_ib;
  F.dt = dt_dev;
  F.nt = flux_nt;
  F.ystride = flux_lmax + 1;
  F.slots = capacity;
  F.stencil = stencil;
  return F;
}

BatchDev Engine::device_view() const {
  BatchDev B;
  B.inst = inst;
  B.ls = ls;
  B.ticket = ticket;
  B.status = status;
  B.E = E_dev;
  B.step = step_dev;
  B.cap = capacity;
  return B;
}

void Engine::build_segment(Segment &sg, const std::vector<int> &act) {
  sg.maxm = 0;
  for (int s : act) sg.maxm = std::max(sg.maxm, spec[s].krylov);
  for (int j = 0; j <= sg.maxm; ++j) {
    // the stencil kernel is launched once per gauge; the elementwise ones once
    std::vector<int> ph, ph_len, ph_vel;
    for (int s : act)
      if (j == 0 || spec[s].krylov > j) {
        ph.push_back(s);
        (spec[s].gauge == TDSE_GAUGE_VELOCITY ? ph_vel : ph_len).push_back(s);
      }
    int off = 0, voff = 0, eoff = 0;
    const int tot = launch_lists(ph_len, kListStencil, off);
    const int vtot = ph_vel.empty() ? 0 : launch_lists(ph_vel, kListStencil, voff);
    const int etot = launch_lists(ph, kListElem, eoff);
    sg.off.push_back(off);
    sg.nact.push_back((int)ph_len.size());
    sg.total.push_back(tot);
    sg.voff.push_back(voff);
    sg.vnact.push_back((int)ph_vel.size());
    sg.vtotal.push_back(vtot);
    sg.eoff.push_back(eoff);
    sg.enact.push_back((int)ph.size());
    sg.etotal.push_back(etot);
  }
  if (ser_cap > 0) {
    sg.dnact = (int)act.size();
    sg.dtotal = launch_lists(act, kListRows, sg.doff);
  }
}

// Upload the staged field table (nE entries) and chunk lists; zero the step counter.
int Engine::upload_run(size_t nE) {
  int rc = ensure(reinterpret_cast<void **>(&E_dev), E_cap, sizeof(double) * std::max<size_t>(1, nE),
                  "field table");
  if (rc) return rc;
  rc = ensure(reinterpret_cast<void **>(&lists), lists_cap, sizeof(int) * std::max<size_t>(1, hlists.size()),
              "chunk lists");
  if (rc) return rc;
  if (!step_dev && cudaMalloc(&step_dev, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    step_dev = nullptr;
    return fail(TDSE_ERR_OOM, "step counter");
  }
  cudaStream_t st = stream;
  if (nE) EN_CUDA(cudaMemcpyAsync(E_dev, hE.data(), sizeof(double) * nE, cudaMemcpyHostToDevice, st), "field upload");
  if (!hlists.empty())
    EN_CUDA(cudaMemcpyAsync(lists, hlists.data(), sizeof(int) * hlists.size(), cudaMemcpyHostToDevice, st),
            "list upload");
  EN_CUDA(cudaMemsetAsync(step_dev, 0, sizeof(int), st), "step counter");
  return TDSE_OK;
}

int Engine::norm_pass(const BatchDev &B, const std::vector<int> &ids, int off, int total) {
  const ChunkList cl = list_at(lists, off, (int)ids.size(), total);
  const unsigned egrid = (unsigned)(sms * sched.eblocks);
  cudaEvent_t pe = prof_begin(TDSE_K_NORM);
  if (precision == TDSE_MIXED) bt_split_mixed<<<egrid, kElemThreads, 0, stream>>>(B, cl);
  else bt_norm_fp64<<<egrid, kElemThreads, 0, stream>>>(B, cl);
  prof_end(pe);
  ++launches;
  EN_CUDA(cudaGetLastError(), "batch norm");
  for (int s : ids) norm_valid[s] = 1;
  return TDSE_OK;
}

int Engine::launch_a(const BatchDev &B, const ChunkList &cl, int j, const Schedule &s) {
  const unsigned grid = (unsigned)(sms * s.sblocks);
  if (precision == TDSE_MIXED) {
    const cudaError_t e = (stencil == 5) ? launch_tile_ring<5>(s.ring, grid, stream, B, cl, j)
                                         : launch_tile_ring<3>(s.ring, grid, stream, B, cl, j);
    EN_CUDA(e, "batch lanczos a (mixed tiles)");
    return TDSE_OK;
  }
  if (stencil == 5) launch_a_st<5>(s.pf, grid, stream, B, cl, j);
  else launch_a_st<3>(s.pf, grid, stream, B, cl, j);
  EN_CUDA(cudaGetLastError(), "batch lanczos a");
  return TDSE_OK;
}

// Velocity-gauge instances: the same FP64 kernel with the (A/c) p_z coupling,
// or the mixed register walker with it.
int Engine::launch_a_velocity(const BatchDev &B, const ChunkList &cl, int j, const Schedule &s) {
  const unsigned grid = (unsigned)(sms * s.sblocks);
  if (precision == TDSE_MIXED) {
    if (stencil == 5) bt_lanczos_a_mixed_vg<5><<<grid, kBlockJ, 0, stream>>>(B, cl, j);
    else bt_lanczos_a_mixed_vg<3><<<grid, kBlockJ, 0, stream>>>(B, cl, j);
    EN_CUDA(cudaGetLastError(), "batch lanczos a (mixed, velocity gauge)");
    return TDSE_OK;
  }
  if (stencil == 5) launch_a_vg_st<5>(s.pf, grid, stream, B, cl, j);
  else launch_a_vg_st<3>(s.pf, grid, stream, B, cl, j);
  EN_CUDA(cudaGetLastError(), "batch lanczos a (velocity gauge)");
  return TDSE_OK;
}

int Engine::launch_b(const BatchDev &B, const ChunkList &cn, int j, const Schedule &s) {
  const unsigned grid = (unsigned)(sms * s.eblocks);
  if (precision == TDSE_MIXED) {
    if (j == 0) bt_lanczos_b_mixed<true><<<grid, kElemThreads, 0, stream>>>(B, cn, j);
    else bt_lanczos_b_mixed<false><<<grid, kElemThreads, 0, stream>>>(B, cn, j);
  } else {
    bt_lanczos_b_fp64<<<grid, kElemThreads, 0, stream>>>(B, cn, j);
  }
  EN_CUDA(cudaGetLastError(), "batch lanczos b");
  return TDSE_OK;
}

// Every launch of one step of a segment; count receives the number of kernels.
int Engine::enqueue_step(const BatchDev &B, const Segment &sg, int &count) {
  count = 0;
  int rc;
  const ChunkList all = list_at(lists, sg.eoff[0], sg.enact[0], sg.etotal[0]);
  for (int j = 0; j < sg.maxm; ++j) {
    const ChunkList cl = list_at(lists, sg.off[j], sg.nact[j], sg.total[j]);
    if (cl.total == 0 && sg.vtotal[j] == 0) break;
    if (cl.total > 0) {
      cudaEvent_t pa = prof_begin(TDSE_K_LANCZOS_A);
      if ((rc = launch_a(B, cl, j, sched))) return rc;
      prof_end(pa);
      ++count;
    }
    if (sg.vtotal[j] > 0) {
      const ChunkList vl = list_at(lists, sg.voff[j], sg.vnact[j], sg.vtotal[j]);
      cudaEvent_t pv = prof_begin(TDSE_K_LANCZOS_A);
      if ((rc = launch_a_velocity(B, vl, j, sched))) return rc;
      prof_end(pv);
      ++count;
    }
    // U_{j+1} only for the instances that go on to iteration j + 1
    if (j + 1 < sg.maxm && sg.etotal[j + 1] > 0) {
      const ChunkList cn = list_at(lists, sg.eoff[j + 1], sg.enact[j + 1], sg.etotal[j + 1]);
      cudaEvent_t pb = prof_begin(TDSE_K_LANCZOS_B);
      if ((rc = launch_b(B, cn, j, sched))) return rc;
      prof_end(pb);
      ++count;
    }
  }
  cudaEvent_t px = prof_begin(TDSE_K_LANCZOS_EXPM);
  EN_CUDA(launch_lanczos_expm_batched(all.nact, all.act, m_dev, dt_dev, run_imag, ls, stream), "batch expm");
  prof_end(px);
  ++count;
  const unsigned egrid = (unsigned)(sms * sched.eblocks);
  cudaEvent_t pc = prof_begin(TDSE_K_LANCZOS_COMBINE);
  if (precision == TDSE_MIXED) {
    if (steps_tab()) bt_combine_mixed<true><<<egrid, kElemThreads, 0, stream>>>(B, all);   // per-step observables read psi
    else bt_combine_mixed<false><<<egrid, kElemThreads, 0, stream>>>(B, all);
  }
  else bt_combine_fp64<<<egrid, kElemThreads, 0, stream>>>(B, all, run_imag ? 0 : 1);
  prof_end(pc);
  ++count;
  EN_CUDA(cudaGetLastError(), "batch combine");
  if (run_imag) {
    cudaEvent_t pn = prof_begin(TDSE_K_NORM);
    bt_imag_normalize<<<egrid, kElemThreads, 0, stream>>>(B, all, dt_dev, imag_e);
    prof_end(pn);
    ++count;
    EN_CUDA(cudaGetLastError(), "batch imaginary-time normalisation");
  }
  if (sg.dtotal > 0 && !run_imag) {
    // the dipole moments of the new states (Sec. 4), recorded per step
    const ChunkList dl = list_at(lists, sg.doff, sg.dnact, sg.dtotal);
    const SeriesDev S = series_view();
    cudaEvent_t pd = prof_begin(TDSE_K_DIPOLE);
    if (stencil == 5) bt_dipole<5><<<egrid, kElemThreads, 0, stream>>>(B, dl, S);
    else bt_dipole<3><<<egrid, kElemThreads, 0, stream>>>(B, dl, S);
    prof_end(pd);
    ++count;
    EN_CUDA(cudaGetLastError(), "batch dipole");
  }
  if (flux_nt >= 0 && !run_imag) {
    // the flux through every instance's sphere and its time integrals (Sec. 4)
    const dim3 fgrid((unsigned)std::max(1, (flux_nt + kFluxThreads / 32 - 1) / (kFluxThreads / 32)),
                     (unsigned)all.nact);
    cudaEvent_t pf = prof_begin(TDSE_K_FLUX);
    bt_flux<<<fgrid, kFluxThreads, sizeof(double2) * 2 * (flux_lmax + 1), stream>>>(B, all.act, flux_view(),
                                                                                     ser_tab, 0);
    prof_end(pf);
    ++count;
    EN_CUDA(cudaGetLastError(), "batch flux");
  }
  bt_next_step<<<1, 1, 0, stream>>>(step_dev);
  ++count;
  EN_CUDA(cudaGetLastError(), "batch step counter");
  return TDSE_OK;
}

int Engine::run(const std::vector<int> &slots, const std::vector<long> &steps, bool imag) {
  if (poisoned) return TDSE_ERR_STATE;
  if (slots.size() != steps.size()) return fail(TDSE_ERR_ARG, "slots and steps differ in length");
  if (imag && precision != TDSE_FP64) return fail(TDSE_ERR_ARG, "imaginary time runs in FP64 batches only");
  long kmax = 0;
  std::vector<char> seen(capacity, 0);
  for (size_t q = 0; q < slots.size(); ++q) {
    const int s = slots[q];
    if (s < 0 || s >= capacity || !placed[s] || steps[q] < 0 || seen[s])
      return fail(TDSE_ERR_ARG, "bad slot or step count");
    seen[s] = 1;
    kmax = std::max(kmax, steps[q]);
  }
  if (kmax == 0) return TDSE_OK;
  if (imag && !imag_e) {
    if (cudaMalloc(&imag_e, sizeof(double) * capacity) != cudaSuccess) {
      cudaGetLastError();
      imag_e = nullptr;
      return fail(TDSE_ERR_OOM, "imaginary-time energies");
    }
    EN_CUDA(cudaMemsetAsync(imag_e, 0xff, sizeof(double) * capacity, stream), "clear energies");   // NaN
  }
  run_imag = imag;
  // launch errors are read with cudaGetLastError: drop an earlier, unrelated
  // non-sticky error of this thread first (a sticky one fails the launches too)
  cudaGetLastError();
  // segments of the run: the active set changes only where a slot finishes
  std::vector<long> ends;
  for (long k : steps)
    if (k > 0) ends.push_back(k);
  std::sort(ends.begin(), ends.end());
  ends.erase(std::unique(ends.begin(), ends.end()), ends.end());
  std::vector<Segment> segs;
  hlists.clear();
  std::vector<int> need_norm;
  for (size_t q = 0; q < slots.size(); ++q)
    if (steps[q] > 0 && !norm_valid[slots[q]]) need_norm.push_back(slots[q]);
  std::sort(need_norm.begin(), need_norm.end());
  int norm_off = 0, norm_total = 0;
  if (!need_norm.empty()) norm_total = launch_lists(need_norm, kListElem, norm_off);
  long n0 = 0;
  for (long e : ends) {
    Segment sg;
    sg.n0 = n0;
    sg.n1 = e;
    std::vector<int> act;
    for (size_t q = 0; q < slots.size(); ++q)
      if (steps[q] >= e) act.push_back(slots[q]);
    std::sort(act.begin(), act.end());
    build_segment(sg, act);
    segs.push_back(std::move(sg));
    n0 = e;
  }
  // field at the mid-point of every step: E[n * capacity + slot]
  const size_t nE = (size_t)kmax * capacity;
  hE.assign(nE, 0.0);
  for (size_t q = 0; q < slots.size() && !imag; ++q) {
    const int s = slots[q];
    const tdse_instance_spec &sp = spec[s];
    for (long n = 0; n < steps[q]; ++n) {
      const double tn = tstart[s] + (double)(nstep[s] + n) * sp.dt;
      hE[(size_t)n * capacity + s] = pulse_at(sp, tn + 0.5 * sp.dt);
    }
  }
  int rc = upload_run(nE);
  if (rc) return rc;
  if (steps_tab() && !imag && (rc = upload_series(slots, steps, nE))) return rc;
  const BatchDev B = device_view();
  if (!need_norm.empty() && (rc = norm_pass(B, need_norm, norm_off, norm_total))) return rc;
  std::vector<std::vector<long long>> eager;
  for (const Segment &sg : segs) {
    const long nst = sg.n1 - sg.n0;
    int count = 0;
    if (profiling) {
      for (long n = 0; n < nst; ++n) {
        if ((rc = enqueue_step(B, sg, count))) return rc;
        launches += count;
      }
      continue;
    }
    std::vector<long long> key = segment_key(sg);
    CachedGraph *hit = nullptr;
    for (CachedGraph &g : graphs)
      if (g.key == key) hit = &g;
    bool repeat = false;
    for (const std::vector<long long> &k : last_eager) repeat = repeat || k == key;
    if (!hit && (nst >= kGraphMinSteps || repeat)) {
      // capture one step and replay it: the step counter on the device selects
      // each step's field
      if (graphs.size() >= kGraphCache) {
        EN_CUDA(cudaStreamSynchronize(stream), "sync before dropping a step graph");
        cudaGraphExecDestroy(graphs.front().exec);
        graphs.erase(graphs.begin());
      }
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      EN_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal), "begin capture");
      rc = enqueue_step(B, sg, count);
      const cudaError_t ec = cudaStreamEndCapture(stream, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      EN_CUDA(ec, "end capture");
      const cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      EN_CUDA(ei, "instantiate step graph");
      graphs.push_back(CachedGraph{std::move(key), ge});
      hit = &graphs.back();
      graph_launches_per_step = count;
      hit->count = count;
    }
    if (hit) {
      for (long n = 0; n < nst; ++n) EN_CUDA(cudaGraphLaunch(hit->exec, stream), "step graph launch");
      launches += (long long)hit->count * nst;
      graph_steps += nst;
    } else {
      for (long n = 0; n < nst; ++n) {
        if ((rc = enqueue_step(B, sg, count))) return rc;
        launches += count;
      }
      eager.push_back(std::move(key));
    }
  }
  last_eager = std::move(eager);
  if (precision == TDSE_MIXED)
    for (size_t q = 0; q < slots.size(); ++q)
      if (steps[q] > 0) psi_stale[slots[q]] = steps_tab() ? 0 : 1;
  for (size_t q = 0; q < slots.size() && !imag; ++q) {
    nstep[slots[q]] += steps[q];
    if (ser_cap > 0) ser_count[slots[q]] = std::min(ser_cap, ser_count[slots[q]] + (long long)steps[q]);
  }
  return TDSE_OK;
}

int Engine::imag_energies(const std::vector<int> &slots, double *out) {
  if (poisoned) return TDSE_ERR_STATE;
  std::vector<double> e(capacity, std::nan(""));
  if (imag_e) {
    EN_CUDA(cudaMemcpyAsync(e.data(), imag_e, sizeof(double) * capacity, cudaMemcpyDeviceToHost, stream),
            "read energies");
  }
  EN_CUDA(cudaStreamSynchronize(stream), "sync energies");
  int rc = check_status();
  if (rc) return rc;
  for (size_t q = 0; q < slots.size(); ++q) out[q] = e[slots[q]];
  return TDSE_OK;
}

// The per-step time table of a run for the dipole series and the flux (t,
// E(t) and A(t)/c at the end of every step) and each slot's series count so far.
int Engine::upload_series(const std::vector<int> &slots, const std::vector<long> &steps, size_t nE) {
  hser_tab.assign(3 * nE, 0.0);
  for (size_t q = 0; q < slots.size(); ++q) {
    const int s = slots[q];
    const tdse_instance_spec &sp = spec[s];
    const PulseParams p{sp.E0, sp.omega, sp.ncycles, sp.cep, sp.pulse_shape};
    const long todo = flux_nt >= 0 ? steps[q] : (long)std::min<long long>(steps[q], ser_cap - ser_count[s]);
    for (long n = 0; n < todo; ++n) {
      const double t = tstart[s] + (double)(nstep[s] + n + 1) * sp.dt;
      double *e = hser_tab.data() + 3 * ((size_t)n * capacity + s);
      e[0] = t;
      e[1] = pulse_field(p, t);
      e[2] = sp.gauge == TDSE_GAUGE_VELOCITY ? pulse_vecpot(p, t) / kLightAU : 0.0;
    }
  }
  int rc = ensure(reinterpret_cast<void **>(&ser_tab), ser_tab_cap, sizeof(double) * std::max<size_t>(3, 3 * nE),
                  "dipole series table");
  if (rc) return rc;
  if (nE)
    EN_CUDA(cudaMemcpyAsync(ser_tab, hser_tab.data(), sizeof(double) * 3 * nE, cudaMemcpyHostToDevice, stream),
            "dipole series table");
  if (ser_cap > 0)
    EN_CUDA(cudaMemcpyAsync(ser_base, ser_count.data(), sizeof(long long) * capacity, cudaMemcpyHostToDevice,
                            stream),
            "dipole series counts");
  return TDSE_OK;
}

int Engine::flux_setup(bool enable, int nt, const double *cos_theta) {
  if (poisoned) return TDSE_ERR_STATE;
  EN_CUDA(cudaStreamSynchronize(stream), "sync before the flux setup");
  cudaFree(flux_state);
  cudaFree(flux_y);
  cudaFree(flux_ct);
  flux_state = flux_y = flux_ct = nullptr;
  flux_nt = -1;
  if (!enable) return TDSE_OK;
  if (nt < 0 || (nt > 0 && !cos_theta)) return fail(TDSE_ERR_ARG, "need ntheta >= 0 and cos_theta for ntheta > 0");
  std::vector<int> ib(capacity, 0), live;
  int lmax = 0;
  for (int s = 0; s < capacity; ++s) {
    if (!placed[s]) continue;
    const tdse_instance_spec &sp = spec[s];
    // the grid point nearest r_b (r_j = (j + 1) dr, j 0-based); a tie goes inwards
    const double x = sp.r_b / sp.dr - 1.0;
    if (!(x > -0.5 && x < (double)sp.N - 0.5)) return fail(TDSE_ERR_ARG, "an instance's r_b lies outside its box");
    ib[s] = std::min(sp.N - 1, std::max(0, (int)std::ceil(x - 0.5)));
    lmax = std::max(lmax, sp.lmax);
    live.push_back(s);
  }
  if (live.empty()) return fail(TDSE_ERR_ARG, "no instance");
  {
    const int rcm = materialize(live);   // the opening flux reads the FP64 states
    if (rcm) return rcm;
  }
  if (sizeof(double2) * 2 * (size_t)(lmax + 1) > 48 * 1024) return fail(TDSE_ERR_ARG, "flux: lmax above 1535");
  // Y_l0(theta_k) = sqrt((2l + 1) / (4 pi)) P_l(cos theta_k), P_l by Bonnet's recurrence
  const size_t ys = (size_t)lmax + 1;
  std::vector<double> ct(nt), y(ys * std::max(nt, 1), 0.0);
  for (int k = 0; k < nt; ++k) {
    const double c = cos_theta[k];
    if (!(c >= -1.0 && c <= 1.0)) return fail(TDSE_ERR_ARG, "cos_theta values must lie in [-1, 1]");
    ct[k] = c;
    double pm = 0.0, p = 1.0;   // P_{l-1}, P_l
    for (int l = 0; l <= lmax; ++l) {
      y[(size_t)k * ys + l] = std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI)) * p;
      const double pn = ((2.0 * l + 1.0) * c * p - (double)l * pm) / (double)(l + 1);
      pm = p;
      p = pn;
    }
  }
  const size_t nstate = (size_t)capacity * (2 + 2 * (size_t)nt);
  const bool ok = cudaMalloc(&flux_state, sizeof(double) * nstate) == cudaSuccess &&
                  cudaMalloc(&flux_y, sizeof(double) * y.size()) == cudaSuccess &&
                  cudaMalloc(&flux_ct, sizeof(double) * std::max(nt, 1)) == cudaSuccess &&
                  (flux_ib || cudaMalloc(&flux_ib, sizeof(int) * capacity) == cudaSuccess) &&
                  (flux_slots || cudaMalloc(&flux_slots, sizeof(int) * capacity) == cudaSuccess);
  if (!ok) {
    cudaGetLastError();
    cudaFree(flux_state);
    cudaFree(flux_y);
    cudaFree(flux_ct);
    flux_state = flux_y = flux_ct = nullptr;
    return fail(TDSE_ERR_OOM, "flux buffers");
  }
  EN_CUDA(cudaMemsetAsync(flux_state, 0, sizeof(double) * nstate, stream), "clear flux");
  EN_CUDA(cudaMemcpyAsync(flux_y, y.data(), sizeof(double) * y.size(), cudaMemcpyHostToDevice, stream), "flux table");
  if (nt) EN_CUDA(cudaMemcpyAsync(flux_ct, ct.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, stream), "angles");
  EN_CUDA(cudaMemcpyAsync(flux_ib, ib.data(), sizeof(int) * capacity, cudaMemcpyHostToDevice, stream), "flux radii");
  EN_CUDA(cudaMemcpyAsync(flux_slots, live.data(), sizeof(int) * live.size(), cudaMemcpyHostToDevice, stream),
          "flux slots");
  flux_nt = nt;
  flux_lmax = lmax;
  // the current states open the integrals at zero: {t, E, A/c} at each slot's time
  std::vector<double> now(3 * (size_t)capacity, 0.0);
  for (int s : live) {
    const tdse_instance_spec &sp = spec[s];
    const PulseParams p{sp.E0, sp.omega, sp.ncycles, sp.cep, sp.pulse_shape};
    const double t = time_of(s);
    now[3 * s] = t;
    now[3 * s + 1] = pulse_field(p, t);
    now[3 * s + 2] = sp.gauge == TDSE_GAUGE_VELOCITY ? pulse_vecpot(p, t) / kLightAU : 0.0;
  }
  int rc = ensure(reinterpret_cast<void **>(&ser_tab), ser_tab_cap, sizeof(double) * now.size(), "flux times");
  if (rc) return rc;
  EN_CUDA(cudaMemcpyAsync(ser_tab, now.data(), sizeof(double) * now.size(), cudaMemcpyHostToDevice, stream),
          "flux times");
  const dim3 fgrid((unsigned)std::max(1, (nt + kFluxThreads / 32 - 1) / (kFluxThreads / 32)), (unsigned)live.size());
  cudaEvent_t pf = prof_begin(TDSE_K_FLUX);
  bt_flux<<<fgrid, kFluxThreads, sizeof(double2) * 2 * (lmax + 1), stream>>>(device_view(), flux_slots, flux_view(),
                                                                             ser_tab, 1);
  prof_end(pf);
  ++launches;
  EN_CUDA(cudaGetLastError(), "flux");
  EN_CUDA(cudaStreamSynchronize(stream), "sync flux setup");
  return TDSE_OK;
}

int Engine::flux_read(int slot, std::vector<double> &out) {
  if (poisoned) return TDSE_ERR_STATE;
  if (slot < 0 || slot >= capacity || !placed[slot]) return fail(TDSE_ERR_ARG, "bad instance");
  if (flux_nt < 0) return fail(TDSE_ERR_ARG, "the flux is not set up");
  const size_t w = 2 + 2 * (size_t)flux_nt;
  out.assign(w, 0.0);
  EN_CUDA(cudaMemcpyAsync(out.data(), flux_state + w * slot, sizeof(double) * w, cudaMemcpyDeviceToHost, stream),
          "read flux");
  EN_CUDA(cudaStreamSynchronize(stream), "sync flux");
  return check_status();
}

int Engine::dipole_series(long long cap) {
  if (poisoned) return TDSE_ERR_STATE;
  if (cap < 0 || cap > (1LL << 40) / (32LL * capacity)) return fail(TDSE_ERR_ARG, "bad dipole series capacity");
  EN_CUDA(cudaStreamSynchronize(stream), "sync before the dipole series");
  cudaFree(ser);
  ser = nullptr;
  ser_cap = 0;
  ser_count.assign(capacity, 0);
  if (cap == 0) return TDSE_OK;
  if (!ser_base && cudaMalloc(&ser_base, sizeof(long long) * capacity) != cudaSuccess) {
    cudaGetLastError();
    ser_base = nullptr;
    return fail(TDSE_ERR_OOM, "dipole series counts");
  }
  if (cudaMalloc(&ser, sizeof(double) * 4 * (size_t)cap * capacity) != cudaSuccess) {
    cudaGetLastError();
    ser = nullptr;
    return fail(TDSE_ERR_OOM, "dipole series");
  }
  ser_cap = cap;
  return TDSE_OK;
}

int Engine::dipole_series_read(int slot, double *out, long long max, long long *count) {
  if (poisoned) return TDSE_ERR_STATE;
  if (slot < 0 || slot >= capacity || !placed[slot]) return fail(TDSE_ERR_ARG, "bad instance");
  const long long n = ser_cap > 0 ? ser_count[slot] : 0;
  if (count) *count = n;
  const long long k = std::min(n, max);
  if (!out || k <= 0) return TDSE_OK;
  EN_CUDA(cudaMemcpyAsync(out, ser + 4 * (size_t)slot * ser_cap, sizeof(double) * 4 * (size_t)k,
                          cudaMemcpyDeviceToHost, stream),
          "read dipole series");
  EN_CUDA(cudaStreamSynchronize(stream), "sync dipole series");
  return check_status();
}

int Engine::set_schedule(const Schedule &s) {
  bool pf_ok = false, ring_ok = false;
  for (int p : kPfChoices) pf_ok = pf_ok || p == s.pf;
  for (int r : kRingChoices) ring_ok = ring_ok || r == s.ring;
  if (!pf_ok || !ring_ok || s.sblocks < 1 || s.sblocks > kTileBlocksPerSM || s.eblocks < 1 ||
      s.eblocks > kElemBlocksPerSM)
    return fail(TDSE_ERR_ARG, "schedule outside the tuned choices");
  sched = s;
  return TDSE_OK;
}

int Engine::autotune(const std::vector<int> &slots) {
  if (poisoned) return TDSE_ERR_STATE;
  std::vector<int> act;
  for (int s : slots) {
    if (s < 0 || s >= capacity || !placed[s]) return fail(TDSE_ERR_ARG, "bad slot");
    act.push_back(s);
  }
  if (act.empty()) return TDSE_OK;
  std::sort(act.begin(), act.end());
  drop_graphs();
  cudaGetLastError();
  hlists.clear();
  std::vector<int> need_norm;
  for (int s : act)
    if (!norm_valid[s]) need_norm.push_back(s);
  int norm_off = 0, norm_total = 0;
  if (!need_norm.empty()) norm_total = launch_lists(need_norm, kListElem, norm_off);
  Segment sg;
  sg.n0 = 0;
  sg.n1 = 1;
  build_segment(sg, act);
  hE.assign((size_t)capacity, 0.0);
  for (int s : act) hE[s] = pulse_at(spec[s], tstart[s] + (double)nstep[s] * spec[s].dt + 0.5 * spec[s].dt);
  int rc = upload_run((size_t)capacity);
  if (rc) return rc;
  const BatchDev B = device_view();
  const bool was_profiling = profiling;
  profiling = false;
  if (!need_norm.empty() && (rc = norm_pass(B, need_norm, norm_off, norm_total))) {
    profiling = was_profiling;
    return rc;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    profiling = was_profiling;
    if (e0) cudaEventDestroy(e0);
    return fail(TDSE_ERR_CUDA, "autotune events");
  }
  // phase 0 launches rewrite only what the next step recomputes (z, U_1 and
  // their scalars), so timing them leaves the state untouched
  const ChunkList a0 = list_at(lists, sg.off[0], sg.nact[0], sg.total[0]);
  const bool have_b = sg.maxm > 1 && sg.etotal[1] > 0;
  const ChunkList b0 = have_b ? list_at(lists, sg.eoff[1], sg.enact[1], sg.etotal[1]) : a0;
  auto time_it = [&](auto &&launch, float &best) -> int {
    best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, stream);
      const int r = launch();
      if (r) return r;
      cudaEventRecord(e1, stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) return fail(TDSE_ERR_CUDA, "autotune sync");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best = std::min(best, ms);
    }
    return TDSE_OK;
  };
  Schedule bestS = sched;
  float bestA = 1e30f, bestB = 1e30f;
  // the staged rows are the mixed tile kernel's
  const int nring = precision == TDSE_MIXED ? (int)(sizeof(kRingChoices) / sizeof(int)) : 1;
  // three blocks per SM only for the mixed tile kernel (the FP64 stencil kernel's blocks fill an SM at two)
  const int sbmax = precision == TDSE_MIXED ? kTileBlocksPerSM : kStencilBlocksPerSM;
  for (int sb = 1; sb <= sbmax && !rc && sg.total[0] > 0; ++sb)
    for (int ri = 0; ri < nring && !rc; ++ri)
      for (int pf : kPfChoices) {
        const int ring = kRingChoices[ri];
        // the mixed tile kernel stages its rows itself: the prefetch distance is the FP64 kernel's
        if (precision == TDSE_MIXED && pf != kPfChoices[0]) continue;
        Schedule c = sched;
        c.pf = pf;
        c.ring = ring;
        c.sblocks = sb;
        float t = 0.f;
        rc = time_it([&]() { return launch_a(B, a0, 0, c); }, t);
        if (rc) break;
        if (t < bestA) {
          bestA = t;
          bestS.pf = pf;
          bestS.ring = ring;
          bestS.sblocks = sb;
        }
      }
  if (!rc && sg.vtotal[0] > 0) {
    // the velocity-gauge instances' phase-0 z, which lanczos_b below reads
    const ChunkList v0 = list_at(lists, sg.voff[0], sg.vnact[0], sg.vtotal[0]);
    rc = launch_a_velocity(B, v0, 0, sched);
  }
  if (!rc && have_b) {
    // lanczos_b at phase 0 reads z from the last A launch above
    for (int eb = 1; eb <= kElemBlocksPerSM && !rc; ++eb) {
      Schedule c = sched;
      c.eblocks = eb;
      float t = 0.f;
      rc = time_it([&]() { return launch_b(B, b0, 0, c); }, t);
      if (!rc && t < bestB) {
        bestB = t;
        bestS.eblocks = eb;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  profiling = was_profiling;
  if (rc) return rc;
  sched = bestS;
  return TDSE_OK;
}

int Engine::observables(int slot, std::vector<double> &out) {
  if (poisoned) return TDSE_ERR_STATE;
  if (slot < 0 || slot >= capacity || !placed[slot]) return fail(TDSE_ERR_ARG, "bad instance");
  {
    const int rcm = materialize({slot});
    if (rcm) return rcm;
  }
  const tdse_instance_spec &s = spec[slot];
  const BatchInst &I = hinst[slot];
  Geometry g;
  g.N = I.N;
  g.L = I.L;
  g.stencil = stencil;
  g.sms = sms;
  g.dr = s.dr;
  g.c0 = g.c1 = g.c2 = 0.0;
  OperatorView op;
  op.diag = I.diag;
  op.rj = I.rj;
  op.kappa = I.kappa;
  op.mask = I.mask;
  op.mask_start = I.mask_start;
  const size_t np = (size_t)5 * observables_blocks(g) * (I.L + 1);
  int rc = ensure(reinterpret_cast<void **>(&obs_partials), obs_cap, sizeof(double) * (np + I.L + 6), "observables");
  if (rc) return rc;
  obs_out = obs_partials + np;
  EN_CUDA(launch_observables(g, op, I.psi, I.ref0, s.r_b, obs_partials, obs_ticket, obs_out, stream), "observables");
  ++launches;
  out.assign(I.L + 5, 0.0);
  EN_CUDA(cudaMemcpyAsync(out.data(), obs_out, sizeof(double) * (I.L + 5), cudaMemcpyDeviceToHost, stream), "read");
  EN_CUDA(cudaStreamSynchronize(stream), "sync");
  rc = check_status();
  if (rc) return rc;
  if (!std::isfinite(out[0])) return fail(TDSE_ERR_NONFINITE, "the instance holds Inf/NaN");
  return TDSE_OK;
}

}  // namespace tdse_dev

// ===========================================================================
// C ABI: a fixed batch
// ===========================================================================
using namespace tdse_dev;

struct tdse_batch {
  Engine eng;
  int count = 0;
  void *mem = nullptr;
  long long npts = 0;
  // pipelined host I/O (tdse_batch_propagate_io): one stream per copy direction
  cudaStream_t io_in = nullptr, io_out = nullptr;
  std::vector<cudaEvent_t> ev;    // ordering events
  std::vector<cudaEvent_t> tev;   // timing events: the input copies, each group's compute
  double io_ratio = 0.0;          // compute time of a point-step over its copy time (0: not yet measured)
  ~tdse_batch() {
    if (eng.stream) cudaStreamSynchronize(eng.stream);
    if (io_in) cudaStreamSynchronize(io_in);
    if (io_out) cudaStreamSynchronize(io_out);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (cudaEvent_t e : tev) cudaEventDestroy(e);
    if (io_in) cudaStreamDestroy(io_in);
    if (io_out) cudaStreamDestroy(io_out);
    cudaFree(mem);
  }
};

namespace {

// Streams, 2 * groups + 1 ordering events and 2 * groups + 2 timing events of
// the pipelined I/O, created once.
int io_ready(tdse_batch *b, int groups) {
  Engine &e = b->eng;
  if (!b->io_in && cudaStreamCreateWithFlags(&b->io_in, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    b->io_in = nullptr;
    return e.fail(TDSE_ERR_CUDA, "I/O stream");
  }
  if (!b->io_out && cudaStreamCreateWithFlags(&b->io_out, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    b->io_out = nullptr;
    return e.fail(TDSE_ERR_CUDA, "I/O stream");
  }
  while ((int)b->ev.size() < 2 * groups + 1) {
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return e.fail(TDSE_ERR_CUDA, "I/O events");
    }
    b->ev.push_back(ev);
  }
  while ((int)b->tev.size() < 2 * groups + 2) {
    cudaEvent_t ev = nullptr;
    if (cudaEventCreate(&ev) != cudaSuccess) {
      cudaGetLastError();
      return e.fail(TDSE_ERR_CUDA, "I/O timing events");
    }
    b->tev.push_back(ev);
  }
  return TDSE_OK;
}

// Taper ratio of the first pipelined call of a batch, before any measurement:
// compute of a point-step over its one-way copy time.  It lies between the two
// precisions' values on the 256-instance batched configuration, as estimated
// from their step and copy times (about 2 mixed, 7 FP64).
constexpr double kIoRatioFirst = 4.0;

}  // namespace

extern "C" {

int tdse_batch_create(const tdse_instance_spec *specs, int count, int stencil, int precision,
                      tdse_batch_t **out) {
  if (!out) return TDSE_ERR_ARG;
  *out = nullptr;
  if (!specs || count < 1 || (stencil != 3 && stencil != 5) ||
      (precision != TDSE_FP64 && precision != TDSE_MIXED))
    return TDSE_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (!valid_spec(specs[i])) return TDSE_ERR_ARG;
  tdse_batch *b = new (std::nothrow) tdse_batch();
  if (!b) return TDSE_ERR_OOM;
  int rc = b->eng.init(count, stencil, precision);
  if (rc) {
    delete b;
    return rc;
  }
  b->count = count;
  std::vector<size_t> at(count);
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    at[i] = total;
    total += instance_bytes(specs[i], precision);
    b->npts += (long long)specs[i].N * (specs[i].lmax + 1);
  }
  if (cudaMalloc(&b->mem, total) != cudaSuccess) {
    cudaGetLastError();
    b->mem = nullptr;
    delete b;
    return TDSE_ERR_OOM;
  }
  for (int i = 0; i < count; ++i) {
    rc = b->eng.place(i, specs[i], static_cast<char *>(b->mem) + at[i]);
    if (rc) {
      delete b;
      return rc;
    }
  }
  *out = b;
  return TDSE_OK;
}

int tdse_batch_destroy(tdse_batch_t *b) {
  delete b;
  return TDSE_OK;
}

const char *tdse_batch_last_error(const tdse_batch_t *b) { return b ? b->eng.err.c_str() : "null batch"; }

int tdse_batch_set_stream(tdse_batch_t *b, void *cuda_stream) {
  return b ? b->eng.set_stream(cuda_stream) : TDSE_ERR_ARG;
}

int tdse_batch_set_state(tdse_batch_t *b, int i, const double *F) {
  return b ? b->eng.set_state(i, F) : TDSE_ERR_ARG;
}

int tdse_batch_get_state(tdse_batch_t *b, int i, double *F) {
  return b ? b->eng.get_state(i, F) : TDSE_ERR_ARG;
}

int tdse_batch_set_states(tdse_batch_t *b, const double *F_all) {
  if (!b) return TDSE_ERR_ARG;
  std::vector<int> slots(b->count);
  for (int i = 0; i < b->count; ++i) slots[i] = i;
  return b->eng.copy_states(slots, const_cast<double *>(F_all), true);
}

int tdse_batch_get_states(tdse_batch_t *b, double *F_all) {
  if (!b) return TDSE_ERR_ARG;
  std::vector<int> slots(b->count);
  for (int i = 0; i < b->count; ++i) slots[i] = i;
  return b->eng.copy_states(slots, F_all, false);
}

double tdse_batch_get_time(const tdse_batch_t *b, int i) {
  return (b && i >= 0 && i < b->count) ? b->eng.time_of(i) : 0.0;
}

int tdse_batch_set_time(tdse_batch_t *b, int i, double t) {
  if (!b) return TDSE_ERR_ARG;
  if (i < 0 || i >= b->count) return b->eng.fail(TDSE_ERR_ARG, "instance index out of range");
  return b->eng.set_time(i, t);
}

int tdse_batch_propagate(tdse_batch_t *b, long nsteps) {
  TraceRange trace("tdse_batch_propagate");
  if (!b) return TDSE_ERR_ARG;
  if (b->eng.poisoned) return TDSE_ERR_STATE;
  if (nsteps < 0) return b->eng.fail(TDSE_ERR_ARG, "nsteps < 0");
  std::vector<int> slots(b->count);
  for (int i = 0; i < b->count; ++i) slots[i] = i;
  return b->eng.run(slots, std::vector<long>(b->count, nsteps));
}

int tdse_batch_propagate_io(tdse_batch_t *b, const double *F_in, double *F_out, long nsteps, int groups) {
  TraceRange trace("tdse_batch_propagate_io");
  if (!b) return TDSE_ERR_ARG;
  Engine &e = b->eng;
  if (e.poisoned) return TDSE_ERR_STATE;
  if (nsteps < 0 || groups < 1) return e.fail(TDSE_ERR_ARG, "need nsteps >= 0 and groups >= 1");
  if (groups > b->count) groups = b->count;
  int rc = io_ready(b, groups);
  if (rc) return rc;
  // each instance's offset in the host buffers (in doubles) and in stencil
  // chunks; contiguous groups (tdse_sched::io_groups) tapered by the compute /
  // copy time ratio that the previous call measured, in whole waves of the
  // stencil grid's warps (one chunk per warp and wave) where the batch allows
  std::vector<size_t> off(b->count + 1, 0), coff(b->count + 1, 0);
  for (int i = 0; i < b->count; ++i) {
    off[i + 1] = off[i] + 2 * (size_t)e.hinst[i].N * (e.hinst[i].L + 1);
    coff[i + 1] = coff[i] + (size_t)e.hinst[i].nchunk;
  }
  const double ratio = (b->io_ratio > 0.0) ? b->io_ratio * (double)std::max(nsteps, 1L) : kIoRatioFirst;
  const size_t wave = (size_t)e.sms * (size_t)e.sched.sblocks * (kBlockJ / 32);
  const std::vector<int> first = tdse_sched::io_groups(coff, groups, ratio, wave);
  auto bytes = [&](int i) { return sizeof(double) * (off[i + 1] - off[i]); };
  // every input copy first, in group order on the input stream, after the
  // work already queued on the compute stream (it may still write the states)
  if (F_in) {
    if (cudaEventRecord(b->ev[2 * groups], e.stream) != cudaSuccess ||
        cudaStreamWaitEvent(b->io_in, b->ev[2 * groups], 0) != cudaSuccess ||
        cudaEventRecord(b->tev[0], b->io_in) != cudaSuccess)
      return e.fail(TDSE_ERR_CUDA, "order input copies");
    for (int g = 0; g < groups; ++g) {
      for (int i = first[g]; i < first[g + 1]; ++i) {
        if (cudaMemcpyAsync(e.hinst[i].psi, F_in + off[i], bytes(i), cudaMemcpyHostToDevice, b->io_in) != cudaSuccess)
          return e.fail(TDSE_ERR_CUDA, "input copy");
        e.norm_valid[i] = 0;
        e.psi_stale[i] = 0;
      }
      if (cudaEventRecord(b->ev[2 * g], b->io_in) != cudaSuccess) return e.fail(TDSE_ERR_CUDA, "input event");
    }
    if (cudaEventRecord(b->tev[1], b->io_in) != cudaSuccess) return e.fail(TDSE_ERR_CUDA, "input event");
  }
  // group g computes once its input is in; its output copy waits for it and
  // overlaps the next group's compute
  for (int g = 0; g < groups; ++g) {
    if (F_in && cudaStreamWaitEvent(e.stream, b->ev[2 * g], 0) != cudaSuccess)
      return e.fail(TDSE_ERR_CUDA, "wait input");
    std::vector<int> slots;
    for (int i = first[g]; i < first[g + 1]; ++i) slots.push_back(i);
    if (cudaEventRecord(b->tev[2 + 2 * g], e.stream) != cudaSuccess) return e.fail(TDSE_ERR_CUDA, "timing event");
    rc = e.run(slots, std::vector<long>(slots.size(), nsteps));
    if (rc) return rc;
    if (F_out && (rc = e.materialize(slots))) return rc;
    if (cudaEventRecord(b->tev[3 + 2 * g], e.stream) != cudaSuccess) return e.fail(TDSE_ERR_CUDA, "timing event");
    if (F_out) {
      if (cudaEventRecord(b->ev[2 * g + 1], e.stream) != cudaSuccess ||
          cudaStreamWaitEvent(b->io_out, b->ev[2 * g + 1], 0) != cudaSuccess)
        return e.fail(TDSE_ERR_CUDA, "output event");
      for (int i = first[g]; i < first[g + 1]; ++i)
        if (cudaMemcpyAsync(F_out + off[i], e.hinst[i].psi, bytes(i), cudaMemcpyDeviceToHost, b->io_out) != cudaSuccess)
          return e.fail(TDSE_ERR_CUDA, "output copy");
    }
  }
  if (cudaStreamSynchronize(b->io_in) != cudaSuccess || cudaStreamSynchronize(e.stream) != cudaSuccess ||
      cudaStreamSynchronize(b->io_out) != cudaSuccess)
    return e.fail(TDSE_ERR_CUDA, "sync I/O");
  // the ratio for the next call: compute time of every group over the copy
  // time of every input, per step
  if (F_in && nsteps > 0) {
    float t_in = 0.f, t_c = 0.f, t = 0.f;
    bool ok = cudaEventElapsedTime(&t_in, b->tev[0], b->tev[1]) == cudaSuccess;
    for (int g = 0; ok && g < groups; ++g) {
      ok = cudaEventElapsedTime(&t, b->tev[2 + 2 * g], b->tev[3 + 2 * g]) == cudaSuccess;
      t_c += t;
    }
    if (!ok) cudaGetLastError();
    else if (t_in > 0.f && t_c > 0.f) b->io_ratio = (double)t_c / ((double)t_in * (double)nsteps);
  }
  return TDSE_OK;
}

int tdse_batch_observables(tdse_batch_t *b, int i, double *norm, double *l_pop, double *dipole,
                           double *yield, double *p_ground) {
  if (!b) return TDSE_ERR_ARG;
  std::vector<double> out;
  const int rc = b->eng.observables(i, out);
  if (rc && rc != TDSE_ERR_NONFINITE) return rc;
  if (norm) *norm = out[0];
  if (dipole) *dipole = out[1];
  if (yield) *yield = out[2];
  if (p_ground) *p_ground = out[3];
  if (l_pop) std::memcpy(l_pop, out.data() + 4, sizeof(double) * (out.size() - 4));
  return rc;
}

int tdse_batch_dipole_series(tdse_batch_t *b, long capacity) {
  return b ? b->eng.dipole_series(capacity) : TDSE_ERR_ARG;
}

int tdse_batch_dipole_series_read(tdse_batch_t *b, int i, double *out, long max_entries, long *count) {
  if (!b || i < 0 || i >= b->count) return TDSE_ERR_ARG;
  long long n = 0;
  const int rc = b->eng.dipole_series_read(i, out, max_entries, &n);
  if (count) *count = (long)n;
  return rc;
}

int tdse_batch_propagate_imag(tdse_batch_t *b, long nsteps, double *energies) {
  if (!b) return TDSE_ERR_ARG;
  if (nsteps < 0) return b->eng.fail(TDSE_ERR_ARG, "nsteps must be >= 0");
  std::vector<int> slots(b->count);
  for (int i = 0; i < b->count; ++i) slots[i] = i;
  int rc = b->eng.run(slots, std::vector<long>(b->count, nsteps), true);
  if (rc || !energies) return rc;
  return b->eng.imag_energies(slots, energies);
}

int tdse_batch_flux_setup(tdse_batch_t *b, int ntheta, const double *cos_theta) {
  if (!b) return TDSE_ERR_ARG;
  return b->eng.flux_setup(ntheta >= 0, ntheta, cos_theta);
}

int tdse_batch_flux_read(tdse_batch_t *b, int i, double *flux, double *yield, double *density, double *pad) {
  if (!b || i < 0 || i >= b->count) return TDSE_ERR_ARG;
  std::vector<double> v;
  const int rc = b->eng.flux_read(i, v);
  if (rc) return rc;
  const size_t nt = (v.size() - 2) / 2;
  if (flux) *flux = v[0];
  if (yield) *yield = v[1];
  if (density && nt) std::memcpy(density, v.data() + 2, sizeof(double) * nt);
  if (pad && nt) std::memcpy(pad, v.data() + 2 + nt, sizeof(double) * nt);
  return TDSE_OK;
}

long long tdse_batch_points(const tdse_batch_t *b) { return b ? b->npts : 0; }
long long tdse_batch_launch_count(const tdse_batch_t *b) { return b ? b->eng.launches : 0; }
long long tdse_batch_graph_steps(const tdse_batch_t *b) { return b ? b->eng.graph_steps : 0; }

int tdse_batch_profile(tdse_batch_t *b, int enable) { return b ? b->eng.profile(enable) : TDSE_ERR_ARG; }

int tdse_batch_autotune(tdse_batch_t *b, tdse_schedule *chosen) {
  if (!b) return TDSE_ERR_ARG;
  std::vector<int> slots(b->count);
  for (int i = 0; i < b->count; ++i) slots[i] = i;
  const int rc = b->eng.autotune(slots);
  if (rc) return rc;
  return tdse_batch_get_schedule(b, chosen);
}

int tdse_batch_set_schedule(tdse_batch_t *b, const tdse_schedule *s) {
  if (!b || !s) return TDSE_ERR_ARG;
  Schedule c;
  c.pf = s->prefetch_rows;
  c.ring = s->ring_rows;
  c.sblocks = s->stencil_blocks_per_sm;
  c.eblocks = s->elem_blocks_per_sm;
  return b->eng.set_schedule(c);
}

int tdse_batch_get_schedule(const tdse_batch_t *b, tdse_schedule *s) {
  if (!b) return TDSE_ERR_ARG;
  if (s) {
    s->prefetch_rows = b->eng.sched.pf;
    s->ring_rows = b->eng.sched.ring;
    s->stencil_blocks_per_sm = b->eng.sched.sblocks;
    s->elem_blocks_per_sm = b->eng.sched.eblocks;
  }
  return TDSE_OK;
}

int tdse_batch_profile_read(tdse_batch_t *b, int kind, double *total_ms, long long *launches) {
  return b ? b->eng.profile_read(kind, total_ms, launches) : TDSE_ERR_ARG;
}

}  // extern "C"
