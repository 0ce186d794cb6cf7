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
#include "tdse_internal.cuh"
#include "tdse_stencil.cuh"

namespace tdse_dev {
namespace {

using namespace common;
using namespace stencil;

constexpr int kChunkSegs = 64;   // 32-point row segments per reduction chunk

struct BatchInst {
  int N, L, m;
  int mask_start;        // first radial index with mask != 1 (N if none)
  long long off;         // first point of the instance in psi / diag / split / z
  long long woff;        // first point of its Krylov area (slot j at woff + j*G)
  int roff;              // first entry in the per-r tables (rj, mask)
  int koff;              // first entry in the kappa table
  int nseg;              // 32-point row segments
  int nchunk;            // reduction chunks
  int cbase;             // first chunk partial slot
  int pad;
  double c1, c2;         // stencil coefficients (c0 is folded into diag)
};

struct BatchDev {
  const BatchInst *inst;
  const double *diag, *rj, *kappa, *mask;
  const float *diagf, *rjf, *kappaf;
  double2 *psi;
  double2 *work;         // FP64 Krylov area: slot 0 = z, slots 1..m-1 = U_j
  float2 *hi, *lo;       // mixed: split of psi
  float2 *mwork;         // mixed Krylov area
  LanczosScalars *ls;
  double *partial;       // chunk partial slots
  unsigned *ticket;      // per-instance arrival counters
  int *status;
  const double *E;       // field of every instance at this step's mid-point
};

struct ChunkList {
  const int *act;        // active instances (ids)
  const int *cpre;       // prefix sums of their chunk counts (nact + 1)
  int nact, total;
};

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
                                           double v, double &total) {
  v = warp_sum(v);
  unsigned last = 0;
  if ((threadIdx.x & 31) == 0) {
    B.partial[I.cbase + ci] = v;
    __threadfence();
    last = (atomicAdd(&B.ticket[inst], 1u) == (unsigned)(I.nchunk - 1)) ? 1u : 0u;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return false;
  __threadfence();
  double s = 0.0;
  for (int c = threadIdx.x & 31; c < I.nchunk; c += 32) s += __ldcg(&B.partial[I.cbase + c]);
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
  in.diag = B.diag + I.off;
  in.rj = B.rj + I.roff;
  in.kappa = B.kappa + I.koff;
  in.N = I.N;
  in.L = I.L;
  in.c1 = I.c1;
  in.c2 = I.c2;
  in.E = B.E[inst];
  return in;
}

template <int ST>
__global__ void __launch_bounds__(kBlockJ, kStencilBlocksPerSM)
    bt_lanczos_a_fp64(BatchDev B, ChunkList cl, int j) {
  for_my_chunks(cl, [&](int inst, int ci) {
    const BatchInst I = B.inst[inst];
    LanczosScalars *ls = B.ls + inst;
    const long long G = (long long)I.N * (I.L + 1);
    const double2 *u = (j == 0) ? B.psi + I.off : B.work + I.woff + (long long)j * G;
    const double2 *up = (j <= 1) ? B.psi + I.off : B.work + I.woff + (long long)(j - 1) * G;
    double2 *z = B.work + I.woff;
    const double sig = ls->sigma[j];
    const double cprev = (j > 0) ? ls->ratio[j] : 0.0;
    const StencilIn in = fp64_in(B, I, inst, u);
    double acc = 0.0;
    chunk_columns(I, ci, [&](int i, int l0, int l1) {
      walk_rows<ST>(in, i, l0, l1, [&](int, size_t idx, double2 t, double2 uc) {
        double2 o;
        if (j > 0) {
          const double2 pv = up[idx];
          o.x = __fma_rn(sig, t.x, __dmul_rn(-cprev, pv.x));
          o.y = __fma_rn(sig, t.y, __dmul_rn(-cprev, pv.y));
        } else {
          o.x = __dmul_rn(sig, t.x);
          o.y = __dmul_rn(sig, t.y);
        }
        z[idx] = o;
        acc = __fma_rn(uc.x, o.x, acc);
        acc = __fma_rn(uc.y, o.y, acc);
      });
    });
    double s;
    if (chunk_done(B, I, inst, ci, acc, s) && (threadIdx.x & 31) == 0) {
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
    const double2 *u = (j == 0) ? B.psi + I.off : B.work + I.woff + (long long)j * G;
    const double2 *z = B.work + I.woff;
    double2 *un = B.work + I.woff + (long long)(j + 1) * G;
    const double c = ls->acoef[j];
    double acc = 0.0;
    chunk_columns(I, ci, [&](int i, int l0, int l1) {
      for (int l = l0; l < l1; ++l) {
        const size_t idx = (size_t)l * I.N + i;
        const double2 zz = z[idx], uu = u[idx];
        const double2 o = make_double2(__fma_rn(c, uu.x, zz.x), __fma_rn(c, uu.y, zz.y));
        un[idx] = o;
        acc = __fma_rn(o.x, o.x, acc);
        acc = __fma_rn(o.y, o.y, acc);
      }
    });
    double s;
    if (chunk_done(B, I, inst, ci, acc, s) && (threadIdx.x & 31) == 0) {
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
    const double2 *x = B.psi + I.off;
    double acc = 0.0;
    chunk_columns(I, ci, [&](int i, int l0, int l1) {
      for (int l = l0; l < l1; ++l) {
        const double2 v = x[(size_t)l * I.N + i];
        acc = __fma_rn(v.x, v.x, acc);
        acc = __fma_rn(v.y, v.y, acc);
      }
    });
    double s;
    if (chunk_done(B, I, inst, ci, acc, s) && (threadIdx.x & 31) == 0) {
      LanczosScalars *ls = B.ls + inst;
      const double nrm = sqrt(s);
      ls->psinorm = nrm;
      ls->sigma[0] = (nrm > 0.0) ? 1.0 / nrm : 0.0;
      if (!isfinite(s)) atomicOr(B.status, kStatusNonFinite);
    }
  });
}

// psi_new = sum_{j<k} coef_j U_j, mask, ||psi_new|| (FP64).
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    bt_combine_fp64(BatchDev B, ChunkList cl) {
  for_my_chunks(cl, [&](int inst, int ci) {
    const BatchInst I = B.inst[inst];
    LanczosScalars *ls = B.ls + inst;
    const long long G = (long long)I.N * (I.L + 1);
    double2 *psi = B.psi + I.off;
    const double2 *U1 = B.work + I.woff + G;
    const double *mask = B.mask + I.roff;
    const int k = ls->kdim;
    double acc = 0.0;
    chunk_columns(I, ci, [&](int i, int l0, int l1) {
      for (int l = l0; l < l1; ++l) {
        const size_t idx = (size_t)l * I.N + i;
        const double2 u0 = psi[idx];
        const double2 c0 = ls->coef[0];
        double ox = __fma_rn(c0.x, u0.x, __dmul_rn(-c0.y, u0.y));
        double oy = __fma_rn(c0.x, u0.y, __dmul_rn(c0.y, u0.x));
        for (int jj = 1; jj < k; ++jj) {
          const double2 u = U1[(size_t)(jj - 1) * G + idx];
          const double2 c = ls->coef[jj];
          ox = __fma_rn(c.x, u.x, ox);
          ox = __fma_rn(-c.y, u.y, ox);
          oy = __fma_rn(c.x, u.y, oy);
          oy = __fma_rn(c.y, u.x, oy);
        }
        if (i >= I.mask_start) {
          const double mv = mask[i];
          ox = __dmul_rn(mv, ox);
          oy = __dmul_rn(mv, oy);
        }
        psi[idx] = make_double2(ox, oy);
        acc = __fma_rn(ox, ox, acc);
        acc = __fma_rn(oy, oy, acc);
      }
    });
    double s;
    if (chunk_done(B, I, inst, ci, acc, s) && (threadIdx.x & 31) == 0) {
      const double nrm = sqrt(s);
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
  in.diag = B.diagf + I.off;
  in.rj = B.rjf + I.roff;
  in.kappa = B.kappaf + I.koff;
  in.N = I.N;
  in.L = I.L;
  in.c1 = (float)I.c1;
  in.c2 = (float)I.c2;
  in.E = (float)B.E[inst];
  return in;
}

template <int ST>
__global__ void __launch_bounds__(kBlockJ, kStencilBlocksPerSM)
    bt_lanczos_a_mixed(BatchDev B, ChunkList cl, int j) {
  for_my_chunks(cl, [&](int inst, int ci) {
    const BatchInst I = B.inst[inst];
    LanczosScalars *ls = B.ls + inst;
    const long long G = (long long)I.N * (I.L + 1);
    const float2 *hi = B.hi + I.off, *lo = B.lo + I.off;
    float2 *z = B.mwork + I.woff;
    const float2 *uprev = (j >= 2) ? B.mwork + I.woff + (long long)(j - 1) * G : nullptr;
    const double sigd = ls->sigma[j];
    const float sig = (float)sigd;
    const float cprev = (j > 0) ? (float)ls->ratio[j] : 0.f;
    float acc = 0.f;
    double accd = 0.0;
    int cnt = 0;
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
      acc = fmaf(u.x, o.x, fmaf(u.y, o.y, acc));
      if (++cnt == 8) {
        accd += (double)acc;
        acc = 0.f;
        cnt = 0;
      }
    };
    if (j == 0) {
      const MixedIn in = mixed_in(B, I, inst, hi, lo, nullptr);
      chunk_columns(I, ci, [&](int i, int l0, int l1) { mixed_walk_rows<ST, true, false>(in, i, l0, l1, epi); });
    } else {
      const MixedIn in = mixed_in(B, I, inst, nullptr, nullptr, B.mwork + I.woff + (long long)j * G);
      chunk_columns(I, ci, [&](int i, int l0, int l1) { mixed_walk_rows<ST, false, true>(in, i, l0, l1, epi); });
    }
    accd += (double)acc;
    double s;
    if (chunk_done(B, I, inst, ci, accd, s) && (threadIdx.x & 31) == 0) {
      ls->alpha[j] = s * sigd;
      ls->acoef[j] = -(s * sigd) * sigd;
    }
  });
}

__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    bt_lanczos_b_mixed(BatchDev B, ChunkList cl, int j) {
  for_my_chunks(cl, [&](int inst, int ci) {
    const BatchInst I = B.inst[inst];
    LanczosScalars *ls = B.ls + inst;
    const long long G = (long long)I.N * (I.L + 1);
    const float2 *u = (j == 0) ? nullptr : B.mwork + I.woff + (long long)j * G;
    const float2 *hi = B.hi + I.off, *lo = B.lo + I.off;
    const float2 *z = B.mwork + I.woff;
    float2 *un = B.mwork + I.woff + (long long)(j + 1) * G;
    const float c = (float)ls->acoef[j];
    float acc = 0.f;
    double accd = 0.0;
    int cnt = 0;
    chunk_columns(I, ci, [&](int i, int l0, int l1) {
      for (int l = l0; l < l1; ++l) {
        const size_t idx = (size_t)l * I.N + i;
        float2 uu;
        if (u) {
          uu = u[idx];
        } else {
          const float2 h = hi[idx], lw = lo[idx];
          uu = make_float2(h.x + lw.x, h.y + lw.y);
        }
        const float2 zz = z[idx];
        const float2 o = make_float2(fmaf(c, uu.x, zz.x), fmaf(c, uu.y, zz.y));
        un[idx] = o;
        acc = fmaf(o.x, o.x, fmaf(o.y, o.y, acc));
        if (++cnt == 8) {
          accd += (double)acc;
          acc = 0.f;
          cnt = 0;
        }
      }
    });
    accd += (double)acc;
    double s;
    if (chunk_done(B, I, inst, ci, accd, s) && (threadIdx.x & 31) == 0) {
      const double beta = sqrt(s);
      ls->beta[j] = beta;
      const double sn = (beta > 0.0) ? 1.0 / beta : 0.0;
      ls->sigma[j + 1] = sn;
      ls->ratio[j + 1] = (sn > 0.0) ? ls->sigma[j] * beta : 0.0;
    }
  });
}

// psi -> (hi, lo) and ||psi|| (FP32 products, FP64 sums).
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    bt_split_mixed(BatchDev B, ChunkList cl) {
  for_my_chunks(cl, [&](int inst, int ci) {
    const BatchInst I = B.inst[inst];
    const double2 *x = B.psi + I.off;
    float2 *hi = B.hi + I.off, *lo = B.lo + I.off;
    float acc = 0.f;
    double accd = 0.0;
    int cnt = 0;
    chunk_columns(I, ci, [&](int i, int l0, int l1) {
      for (int l = l0; l < l1; ++l) {
        const size_t idx = (size_t)l * I.N + i;
        float2 h, lw;
        split2(x[idx], h, lw);
        hi[idx] = h;
        lo[idx] = lw;
        acc = fmaf(h.x, h.x, fmaf(h.y, h.y, acc));
        if (++cnt == 8) {
          accd += (double)acc;
          acc = 0.f;
          cnt = 0;
        }
      }
    });
    accd += (double)acc;
    double s;
    if (chunk_done(B, I, inst, ci, accd, s) && (threadIdx.x & 31) == 0) {
      LanczosScalars *ls = B.ls + inst;
      const double nrm = sqrt(s);
      ls->psinorm = nrm;
      ls->sigma[0] = (nrm > 0.0) ? 1.0 / nrm : 0.0;
      if (!isfinite(s)) atomicOr(B.status, kStatusNonFinite);
    }
  });
}

// psi_new = coef_0 psi (FP64) + sum_{j>=1} coef_j U_j (FP32, added in FP64),
// mask, split, ||psi_new||.
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    bt_combine_mixed(BatchDev B, ChunkList cl) {
  for_my_chunks(cl, [&](int inst, int ci) {
    const BatchInst I = B.inst[inst];
    LanczosScalars *ls = B.ls + inst;
    const long long G = (long long)I.N * (I.L + 1);
    double2 *psi = B.psi + I.off;
    float2 *hi = B.hi + I.off, *lo = B.lo + I.off;
    const float2 *U1 = B.mwork + I.woff + G;
    const double *mask = B.mask + I.roff;
    const int k = ls->kdim;
    const double2 c0 = ls->coef[0];
    float acc = 0.f;
    double accd = 0.0;
    int cnt = 0;
    chunk_columns(I, ci, [&](int i, int l0, int l1) {
      for (int l = l0; l < l1; ++l) {
        const size_t idx = (size_t)l * I.N + i;
        float cx = 0.f, cy = 0.f;
        for (int jj = 1; jj < k; ++jj) {
          const float2 u = U1[(size_t)(jj - 1) * G + idx];
          const double2 cd = ls->coef[jj];
          const float2 c = make_float2((float)cd.x, (float)cd.y);
          cx = fmaf(c.x, u.x, cx);
          cx = fmaf(-c.y, u.y, cx);
          cy = fmaf(c.x, u.y, cy);
          cy = fmaf(c.y, u.x, cy);
        }
        const double2 p = psi[idx];
        double ox = fma(c0.x, p.x, fma(-c0.y, p.y, (double)cx));
        double oy = fma(c0.x, p.y, fma(c0.y, p.x, (double)cy));
        if (i >= I.mask_start) {
          const double mv = mask[i];
          ox *= mv;
          oy *= mv;
        }
        const double2 o = make_double2(ox, oy);
        psi[idx] = o;
        float2 h, lw;
        split2(o, h, lw);
        hi[idx] = h;
        lo[idx] = lw;
        acc = fmaf(h.x, h.x, fmaf(h.y, h.y, acc));
        if (++cnt == 8) {
          accd += (double)acc;
          acc = 0.f;
          cnt = 0;
        }
      }
    });
    accd += (double)acc;
    double s;
    if (chunk_done(B, I, inst, ci, accd, s) && (threadIdx.x & 31) == 0) {
      const double nrm = sqrt(s);
      ls->psinorm = nrm;
      ls->sigma[0] = (nrm > 0.0) ? 1.0 / nrm : 0.0;
      if (!isfinite(s)) atomicOr(B.status, kStatusNonFinite);
    }
  });
}

}  // namespace
}  // namespace tdse_dev

// ===========================================================================
// Host side
// ===========================================================================
using namespace tdse_dev;

struct tdse_batch {
  int count = 0, stencil = 5, precision = TDSE_FP64;
  std::vector<tdse_instance_spec> spec;
  std::vector<BatchInst> hinst;
  std::vector<double> t;             // time of every instance
  long long npts = 0, nwork = 0;
  int nchunks = 0, max_m = 0, sms = 0;
  cudaStream_t own_stream = nullptr, stream = nullptr;
  // device
  BatchInst *inst = nullptr;
  double *diag = nullptr, *rj = nullptr, *kappa = nullptr, *mask = nullptr;
  float *diagf = nullptr, *rjf = nullptr, *kappaf = nullptr;
  double2 *psi = nullptr, *work = nullptr;
  float2 *split = nullptr, *mwork = nullptr;
  LanczosScalars *ls = nullptr;
  double *partial = nullptr;
  unsigned *ticket = nullptr;
  int *status = nullptr;
  int *act = nullptr, *cpre = nullptr;   // active lists of every phase, flattened
  int *m_dev = nullptr;
  double *dt_dev = nullptr, *E_dev = nullptr;
  long long E_cap = 0;
  std::vector<int> act_off, act_n, act_total;   // per phase j (0..max_m)
  double *obs_partials = nullptr, *obs_out = nullptr, *obs_rj = nullptr, *obs_kappa = nullptr;
  double2 *ref0 = nullptr;
  bool norm_valid = false;
  long long launches = 0;
  std::string err;
  bool poisoned = false;
  // per-kernel timing (tdse_batch_profile)
  bool profiling = false;
  struct Mark { int kind; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  size_t nmarks = 0;
  double prof_ms[TDSE_K_COUNT] = {0};
  long long prof_n[TDSE_K_COUNT] = {0};
};

namespace {

int bfail(tdse_batch *b, int code, const std::string &msg) {
  if (b) {
    b->err = msg;
    if (code == TDSE_ERR_CUDA) b->poisoned = true;
  }
  return code;
}

#define BT_CUDA(b, call, what)                                                        \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return bfail(b, TDSE_ERR_CUDA, std::string(what) + ": " + \
                                                              cudaGetErrorString(e_)); \
  } while (0)

// Start event of a profiled launch; returns the stop event to record after it.
cudaEvent_t bprof_begin(tdse_batch *b, int kind) {
  if (!b->profiling) return nullptr;
  if (b->nmarks == b->marks.size()) {
    tdse_batch::Mark m;
    if (cudaEventCreate(&m.a) != cudaSuccess || cudaEventCreate(&m.b) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    b->marks.push_back(m);
  }
  tdse_batch::Mark &m = b->marks[b->nmarks++];
  m.kind = kind;
  cudaEventRecord(m.a, b->stream);
  return m.b;
}

void bprof_end(tdse_batch *b, cudaEvent_t e) {
  if (e) cudaEventRecord(e, b->stream);
}

int bprof_collect(tdse_batch *b) {
  BT_CUDA(b, cudaStreamSynchronize(b->stream), "sync profile");
  for (size_t i = 0; i < b->nmarks; ++i) {
    float ms = 0.f;
    BT_CUDA(b, cudaEventElapsedTime(&ms, b->marks[i].a, b->marks[i].b), "event time");
    b->prof_ms[b->marks[i].kind] += ms;
    b->prof_n[b->marks[i].kind] += 1;
  }
  b->nmarks = 0;
  return TDSE_OK;
}

double pulse_at(const tdse_instance_spec &s, double t) {
  if (s.E0 == 0.0 || s.omega <= 0.0) return 0.0;
  const double T = 2.0 * M_PI * s.ncycles / s.omega;
  if (t < 0.0 || t > T) return 0.0;
  const double env = std::sin(M_PI * t / T);
  return s.E0 * env * env * std::sin(s.omega * t + s.cep);
}

void bfree(tdse_batch *b) {
  cudaFree(b->inst);
  cudaFree(b->diag);
  cudaFree(b->rj);
  cudaFree(b->kappa);
  cudaFree(b->mask);
  cudaFree(b->diagf);
  cudaFree(b->rjf);
  cudaFree(b->kappaf);
  cudaFree(b->psi);
  cudaFree(b->work);
  cudaFree(b->split);
  cudaFree(b->mwork);
  cudaFree(b->ls);
  cudaFree(b->partial);
  cudaFree(b->ticket);
  cudaFree(b->status);
  cudaFree(b->act);
  cudaFree(b->cpre);
  cudaFree(b->m_dev);
  cudaFree(b->dt_dev);
  cudaFree(b->E_dev);
  cudaFree(b->obs_partials);
  cudaFree(b->obs_out);
  cudaFree(b->ref0);
  for (auto &m : b->marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
}

BatchDev dev_view(const tdse_batch *b) {
  BatchDev B;
  B.inst = b->inst;
  B.diag = b->diag;
  B.rj = b->rj;
  B.kappa = b->kappa;
  B.mask = b->mask;
  B.diagf = b->diagf;
  B.rjf = b->rjf;
  B.kappaf = b->kappaf;
  B.psi = b->psi;
  B.work = b->work;
  B.hi = b->split;
  B.lo = b->split ? b->split + b->npts : nullptr;
  B.mwork = b->mwork;
  B.ls = b->ls;
  B.partial = b->partial;
  B.ticket = b->ticket;
  B.status = b->status;
  B.E = b->E_dev;
  return B;
}

ChunkList chunk_list(const tdse_batch *b, int j) {
  ChunkList cl;
  cl.act = b->act + b->act_off[j];
  cl.cpre = b->cpre + b->act_off[j] + j;   // prefix arrays have nact + 1 entries
  cl.nact = b->act_n[j];
  cl.total = b->act_total[j];
  return cl;
}

bool valid_spec(const tdse_instance_spec &s) {
  if (s.N < 1 || s.lmax < 0 || !(s.dr > 0.0) || !(s.dt > 0.0) || !std::isfinite(s.Z)) return false;
  if (s.krylov < 1 || s.krylov > TDSE_MAX_KRYLOV) return false;
  if (!std::isfinite(s.E0) || !std::isfinite(s.omega) || !std::isfinite(s.ncycles) ||
      !std::isfinite(s.cep) || !std::isfinite(s.absorber_r) || !std::isfinite(s.r_b))
    return false;
  if (s.E0 != 0.0 && (!(s.omega > 0.0) || !(s.ncycles > 0.0))) return false;
  return true;
}

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
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return TDSE_ERR_CUDA;
  }
  tdse_batch *b = new (std::nothrow) tdse_batch();
  if (!b) return TDSE_ERR_OOM;
  b->count = count;
  b->stencil = stencil;
  b->precision = precision;
  b->sms = sms;
  b->spec.assign(specs, specs + count);
  b->t.assign(count, 0.0);
  // layout
  long long off = 0, woff = 0;
  int roff = 0, koff = 0, cbase = 0, maxm = 0;
  b->hinst.resize(count);
  for (int i = 0; i < count; ++i) {
    const tdse_instance_spec &s = specs[i];
    BatchInst &I = b->hinst[i];
    const long long G = (long long)s.N * (s.lmax + 1);
    I.N = s.N;
    I.L = s.lmax;
    I.m = s.krylov;
    I.off = off;
    I.woff = woff;
    I.roff = roff;
    I.koff = koff;
    const long long nseg = (long long)((s.N + 31) / 32) * (s.lmax + 1);
    if (nseg > (1LL << 30) || off + G > (1LL << 40)) {
      delete b;
      return TDSE_ERR_ARG;
    }
    I.nseg = (int)nseg;
    I.nchunk = (int)((nseg + kChunkSegs - 1) / kChunkSegs);
    I.cbase = cbase;
    I.pad = 0;
    const double h2 = s.dr * s.dr;
    if (stencil == 5) {
      I.c1 = -16.0 / (24.0 * h2);
      I.c2 = 1.0 / (24.0 * h2);
    } else {
      I.c1 = -0.5 / h2;
      I.c2 = 0.0;
    }
    off += G;
    woff += G * s.krylov;
    roff += s.N;
    koff += s.lmax + 2;
    cbase += I.nchunk;
    maxm = std::max(maxm, s.krylov);
  }
  b->npts = off;
  b->nwork = woff;
  b->nchunks = cbase;
  b->max_m = maxm;
  // host tables
  std::vector<double> diag(off), rj(roff), kap(koff), msk(roff, 1.0);
  std::vector<double> psi0(2 * off, 0.0);
  for (int i = 0; i < count; ++i) {
    const tdse_instance_spec &s = specs[i];
    BatchInst &I = b->hinst[i];
    const double c0 = (stencil == 5) ? 30.0 / (24.0 * s.dr * s.dr) : 1.0 / (s.dr * s.dr);
    for (int j = 0; j < s.N; ++j) rj[I.roff + j] = (double)(j + 1) * s.dr;
    for (int l = 0; l <= s.lmax; ++l) {
      const double cent = 0.5 * (double)l * (double)(l + 1);
      for (int j = 0; j < s.N; ++j) {
        const double r = rj[I.roff + j];
        diag[I.off + (long long)l * s.N + j] = c0 + cent / (r * r) - s.Z / r;
      }
    }
    kap[I.koff] = 0.0;
    for (int l = 1; l <= s.lmax; ++l) {
      const double ll = (double)l * (double)l;
      kap[I.koff + l] = std::sqrt(ll / (4.0 * ll - 1.0));
    }
    kap[I.koff + s.lmax + 1] = 0.0;
    I.mask_start = s.N;
    const double R = rj[I.roff + s.N - 1], ra = s.absorber_r;
    if (ra < R) {
      for (int j = 0; j < s.N; ++j) {
        const double r = rj[I.roff + j];
        if (r > ra) {
          if (I.mask_start == s.N) I.mask_start = j;
          msk[I.roff + j] = std::pow(std::cos(0.5 * M_PI * (r - ra) / (R - ra)), 0.125);
        }
      }
    }
    // normalised 1s state in l = 0
    double nrm = 0.0;
    for (int j = 0; j < s.N; ++j) {
      const double r = rj[I.roff + j];
      const double p = 2.0 * r * std::exp(-r);
      psi0[2 * (I.off + j)] = p;
      nrm += p * p;
    }
    const double sc = 1.0 / std::sqrt(s.dr * nrm);
    for (int j = 0; j < s.N; ++j) psi0[2 * (I.off + j)] *= sc;
  }
  // active lists: phase j holds the instances with krylov > j
  std::vector<int> act, cpre;
  b->act_off.resize(maxm + 1);
  b->act_n.resize(maxm + 1);
  b->act_total.resize(maxm + 1);
  for (int j = 0; j <= maxm; ++j) {
    b->act_off[j] = (int)act.size();
    int n = 0, tot = 0;
    std::vector<int> pre;
    pre.push_back(0);
    for (int i = 0; i < count; ++i) {
      if (specs[i].krylov > j || j == 0) {
        act.push_back(i);
        tot += b->hinst[i].nchunk;
        pre.push_back(tot);
        ++n;
      }
    }
    // cpre is stored with one extra entry per phase: offset act_off[j] + j
    while ((int)cpre.size() < b->act_off[j] + j) cpre.push_back(0);
    cpre.insert(cpre.end(), pre.begin(), pre.end());
    b->act_n[j] = n;
    b->act_total[j] = tot;
  }
  std::vector<int> mh(count);
  std::vector<double> dth(count);
  for (int i = 0; i < count; ++i) {
    mh[i] = specs[i].krylov;
    dth[i] = specs[i].dt;
  }
  // device allocation
  if (cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    b->own_stream = nullptr;
    delete b;
    return TDSE_ERR_CUDA;
  }
  b->stream = b->own_stream;
  int maxL = 0, maxN = 0;
  for (int i = 0; i < count; ++i) {
    maxL = std::max(maxL, specs[i].lmax);
    maxN = std::max(maxN, specs[i].N);
  }
  const bool mixed = precision == TDSE_MIXED;
  bool ok = cudaMalloc(&b->inst, sizeof(BatchInst) * count) == cudaSuccess &&
            cudaMalloc(&b->diag, sizeof(double) * off) == cudaSuccess &&
            cudaMalloc(&b->rj, sizeof(double) * roff) == cudaSuccess &&
            cudaMalloc(&b->kappa, sizeof(double) * koff) == cudaSuccess &&
            cudaMalloc(&b->mask, sizeof(double) * roff) == cudaSuccess &&
            cudaMalloc(&b->psi, sizeof(double2) * off) == cudaSuccess &&
            cudaMalloc(&b->ls, sizeof(LanczosScalars) * count) == cudaSuccess &&
            cudaMalloc(&b->partial, sizeof(double) * std::max(1, cbase)) == cudaSuccess &&
            cudaMalloc(&b->ticket, sizeof(unsigned) * count) == cudaSuccess &&
            cudaMalloc(&b->status, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&b->act, sizeof(int) * std::max<size_t>(1, act.size())) == cudaSuccess &&
            cudaMalloc(&b->cpre, sizeof(int) * std::max<size_t>(1, cpre.size())) == cudaSuccess &&
            cudaMalloc(&b->m_dev, sizeof(int) * count) == cudaSuccess &&
            cudaMalloc(&b->dt_dev, sizeof(double) * count) == cudaSuccess &&
            cudaMalloc(&b->obs_partials, sizeof(double) * ((size_t)5 * 8 * (maxL + 1) + 2)) == cudaSuccess &&
            cudaMalloc(&b->obs_out, sizeof(double) * (maxL + 6)) == cudaSuccess &&
            cudaMalloc(&b->ref0, sizeof(double2) * maxN) == cudaSuccess;
  if (ok && !mixed) ok = cudaMalloc(&b->work, sizeof(double2) * woff) == cudaSuccess;
  if (ok && mixed)
    ok = cudaMalloc(&b->diagf, sizeof(float) * off) == cudaSuccess &&
         cudaMalloc(&b->rjf, sizeof(float) * roff) == cudaSuccess &&
         cudaMalloc(&b->kappaf, sizeof(float) * koff) == cudaSuccess &&
         cudaMalloc(&b->split, sizeof(float2) * off * 2) == cudaSuccess &&
         cudaMalloc(&b->mwork, sizeof(float2) * woff) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    bfree(b);
    delete b;
    return TDSE_ERR_OOM;
  }
  cudaStream_t s = b->stream;
  bool cp = cudaMemcpyAsync(b->inst, b->hinst.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(b->diag, diag.data(), sizeof(double) * off, cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(b->rj, rj.data(), sizeof(double) * roff, cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(b->kappa, kap.data(), sizeof(double) * koff, cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(b->mask, msk.data(), sizeof(double) * roff, cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(b->psi, psi0.data(), sizeof(double) * 2 * off, cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemsetAsync(b->ls, 0, sizeof(LanczosScalars) * count, s) == cudaSuccess &&
            cudaMemsetAsync(b->ticket, 0, sizeof(unsigned) * count, s) == cudaSuccess &&
            cudaMemsetAsync(b->status, 0, sizeof(int), s) == cudaSuccess &&
            cudaMemcpyAsync(b->act, act.data(), sizeof(int) * act.size(), cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(b->cpre, cpre.data(), sizeof(int) * cpre.size(), cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(b->m_dev, mh.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(b->dt_dev, dth.data(), sizeof(double) * count, cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemsetAsync(b->obs_partials, 0, sizeof(double) * ((size_t)5 * 8 * (maxL + 1) + 2), s) == cudaSuccess;
  if (cp && mixed) {
    std::vector<float> df(off), rf(roff), kf(koff);
    for (int i = 0; i < count; ++i) {
      const tdse_instance_spec &sp = specs[i];
      const BatchInst &I = b->hinst[i];
      const double c0 = (stencil == 5) ? 30.0 / (24.0 * sp.dr * sp.dr) : 1.0 / (sp.dr * sp.dr);
      const long long G = (long long)sp.N * (sp.lmax + 1);
      for (long long q = 0; q < G; ++q) df[I.off + q] = (float)(diag[I.off + q] - c0);
    }
    for (int q = 0; q < roff; ++q) rf[q] = (float)rj[q];
    for (int q = 0; q < koff; ++q) kf[q] = (float)kap[q];
    cp = cudaMemcpyAsync(b->diagf, df.data(), sizeof(float) * off, cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaMemcpyAsync(b->rjf, rf.data(), sizeof(float) * roff, cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaMemcpyAsync(b->kappaf, kf.data(), sizeof(float) * koff, cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaStreamSynchronize(s) == cudaSuccess;
  }
  if (!cp || cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    bfree(b);
    delete b;
    return TDSE_ERR_CUDA;
  }
  *out = b;
  return TDSE_OK;
}

int tdse_batch_destroy(tdse_batch_t *b) {
  if (!b) return TDSE_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  bfree(b);
  delete b;
  return TDSE_OK;
}

const char *tdse_batch_last_error(const tdse_batch_t *b) { return b ? b->err.c_str() : "null batch"; }

int tdse_batch_set_stream(tdse_batch_t *b, void *cuda_stream) {
  if (!b) return TDSE_ERR_ARG;
  if (b->poisoned) return TDSE_ERR_STATE;
  BT_CUDA(b, cudaStreamSynchronize(b->stream), "sync");
  b->stream = cuda_stream ? (cudaStream_t)cuda_stream : b->own_stream;
  return TDSE_OK;
}

int tdse_batch_set_state(tdse_batch_t *b, int i, const double *F) {
  if (!b) return TDSE_ERR_ARG;
  if (b->poisoned) return TDSE_ERR_STATE;
  if (i < 0 || i >= b->count || !F) return bfail(b, TDSE_ERR_ARG, "bad instance or null state");
  const BatchInst &I = b->hinst[i];
  const size_t G = (size_t)I.N * (I.L + 1);
  BT_CUDA(b, cudaMemcpyAsync(b->psi + I.off, F, sizeof(double2) * G, cudaMemcpyHostToDevice, b->stream), "set state");
  BT_CUDA(b, cudaStreamSynchronize(b->stream), "sync");
  b->norm_valid = false;
  return TDSE_OK;
}

int tdse_batch_get_state(tdse_batch_t *b, int i, double *F) {
  if (!b) return TDSE_ERR_ARG;
  if (b->poisoned) return TDSE_ERR_STATE;
  if (i < 0 || i >= b->count || !F) return bfail(b, TDSE_ERR_ARG, "bad instance or null state");
  const BatchInst &I = b->hinst[i];
  const size_t G = (size_t)I.N * (I.L + 1);
  BT_CUDA(b, cudaMemcpyAsync(F, b->psi + I.off, sizeof(double2) * G, cudaMemcpyDeviceToHost, b->stream), "get state");
  BT_CUDA(b, cudaStreamSynchronize(b->stream), "sync");
  return TDSE_OK;
}

double tdse_batch_get_time(const tdse_batch_t *b, int i) {
  return (b && i >= 0 && i < b->count) ? b->t[i] : 0.0;
}

int tdse_batch_propagate(tdse_batch_t *b, long nsteps) {
  if (!b) return TDSE_ERR_ARG;
  if (b->poisoned) return TDSE_ERR_STATE;
  if (nsteps < 0) return bfail(b, TDSE_ERR_ARG, "nsteps < 0");
  if (nsteps == 0) return TDSE_OK;
  const int C = b->count;
  // field of every instance at the mid-point of every step of this call
  const long long nE = (long long)nsteps * C;
  if (nE > b->E_cap) {
    BT_CUDA(b, cudaStreamSynchronize(b->stream), "sync");
    cudaFree(b->E_dev);
    b->E_dev = nullptr;
    b->E_cap = 0;
    if (cudaMalloc(&b->E_dev, sizeof(double) * nE) != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, TDSE_ERR_OOM, "field table");
    }
    b->E_cap = nE;
  }
  std::vector<double> Eh(nE);
  for (long n = 0; n < nsteps; ++n)
    for (int i = 0; i < C; ++i)
      Eh[(size_t)n * C + i] = pulse_at(b->spec[i], b->t[i] + (double)n * b->spec[i].dt + 0.5 * b->spec[i].dt);
  BT_CUDA(b, cudaMemcpyAsync(b->E_dev, Eh.data(), sizeof(double) * nE, cudaMemcpyHostToDevice, b->stream), "field upload");
  BT_CUDA(b, cudaStreamSynchronize(b->stream), "sync field upload");
  const bool mixed = b->precision == TDSE_MIXED;
  const unsigned sgrid = (unsigned)(b->sms * kStencilBlocksPerSM);
  const unsigned egrid = (unsigned)(b->sms * kElemBlocksPerSM);
  cudaStream_t st = b->stream;
  BatchDev B = dev_view(b);
  const ChunkList all = chunk_list(b, 0);
  if (!b->norm_valid) {
    cudaEvent_t pe = bprof_begin(b, TDSE_K_NORM);
    if (mixed) bt_split_mixed<<<egrid, kElemThreads, 0, st>>>(B, all);
    else bt_norm_fp64<<<egrid, kElemThreads, 0, st>>>(B, all);
    bprof_end(b, pe);
    ++b->launches;
    BT_CUDA(b, cudaGetLastError(), "batch norm");
  }
  for (long n = 0; n < nsteps; ++n) {
    B.E = b->E_dev + (size_t)n * C;
    for (int j = 0; j < b->max_m; ++j) {
      const ChunkList cl = chunk_list(b, j);
      if (cl.total == 0) break;
      cudaEvent_t pa = bprof_begin(b, TDSE_K_LANCZOS_A);
      if (mixed) {
        if (b->stencil == 5) bt_lanczos_a_mixed<5><<<sgrid, kBlockJ, 0, st>>>(B, cl, j);
        else bt_lanczos_a_mixed<3><<<sgrid, kBlockJ, 0, st>>>(B, cl, j);
      } else {
        if (b->stencil == 5) bt_lanczos_a_fp64<5><<<sgrid, kBlockJ, 0, st>>>(B, cl, j);
        else bt_lanczos_a_fp64<3><<<sgrid, kBlockJ, 0, st>>>(B, cl, j);
      }
      bprof_end(b, pa);
      ++b->launches;
      BT_CUDA(b, cudaGetLastError(), "batch lanczos a");
      // U_{j+1} only for the instances that go on to iteration j + 1
      const ChunkList cn = chunk_list(b, j + 1);
      if (j + 1 < b->max_m && cn.total > 0) {
        cudaEvent_t pb = bprof_begin(b, TDSE_K_LANCZOS_B);
        if (mixed) bt_lanczos_b_mixed<<<egrid, kElemThreads, 0, st>>>(B, cn, j);
        else bt_lanczos_b_fp64<<<egrid, kElemThreads, 0, st>>>(B, cn, j);
        bprof_end(b, pb);
        ++b->launches;
        BT_CUDA(b, cudaGetLastError(), "batch lanczos b");
      }
    }
    cudaEvent_t px = bprof_begin(b, TDSE_K_LANCZOS_EXPM);
    BT_CUDA(b, launch_lanczos_expm_batched(C, b->m_dev, b->dt_dev, b->ls, st), "batch expm");
    bprof_end(b, px);
    ++b->launches;
    cudaEvent_t pc = bprof_begin(b, TDSE_K_LANCZOS_COMBINE);
    if (mixed) bt_combine_mixed<<<egrid, kElemThreads, 0, st>>>(B, all);
    else bt_combine_fp64<<<egrid, kElemThreads, 0, st>>>(B, all);
    bprof_end(b, pc);
    ++b->launches;
    BT_CUDA(b, cudaGetLastError(), "batch combine");
  }
  for (int i = 0; i < C; ++i) b->t[i] += (double)nsteps * b->spec[i].dt;
  b->norm_valid = true;
  return TDSE_OK;
}

int tdse_batch_observables(tdse_batch_t *b, int i, double *norm, double *l_pop, double *dipole,
                           double *yield, double *p_ground) {
  if (!b) return TDSE_ERR_ARG;
  if (b->poisoned) return TDSE_ERR_STATE;
  if (i < 0 || i >= b->count) return bfail(b, TDSE_ERR_ARG, "bad instance");
  const tdse_instance_spec &s = b->spec[i];
  const BatchInst &I = b->hinst[i];
  Geometry g;
  g.N = I.N;
  g.L = I.L;
  g.stencil = b->stencil;
  g.sms = b->sms;
  g.dr = s.dr;
  g.c0 = g.c1 = g.c2 = 0.0;
  OperatorView op;
  op.diag = b->diag + I.off;
  op.rj = b->rj + I.roff;
  op.kappa = b->kappa + I.koff;
  op.mask = b->mask + I.roff;
  op.mask_start = I.mask_start;
  // reference of p_ground: the 1s state of the instance's grid
  std::vector<double> ref(2 * (size_t)I.N, 0.0);
  double nrm = 0.0;
  for (int j = 0; j < I.N; ++j) {
    const double r = (double)(j + 1) * s.dr;
    ref[2 * j] = 2.0 * r * std::exp(-r);
    nrm += ref[2 * j] * ref[2 * j];
  }
  for (int j = 0; j < I.N; ++j) ref[2 * j] /= std::sqrt(s.dr * nrm);
  BT_CUDA(b, cudaMemcpyAsync(b->ref0, ref.data(), sizeof(double) * ref.size(), cudaMemcpyHostToDevice, b->stream), "ref");
  // the counter sits after the largest partial block, at the same address for every instance
  int maxL = 0;
  for (const auto &sp : b->spec) maxL = std::max(maxL, sp.lmax);
  unsigned *ticket = reinterpret_cast<unsigned *>(b->obs_partials + (size_t)5 * 8 * (maxL + 1));
  BT_CUDA(b, launch_observables(g, op, b->psi + I.off, b->ref0, s.r_b, b->obs_partials, ticket, b->obs_out,
                                b->stream),
          "observables");
  ++b->launches;
  std::vector<double> out(I.L + 5);
  BT_CUDA(b, cudaMemcpyAsync(out.data(), b->obs_out, sizeof(double) * (I.L + 5), cudaMemcpyDeviceToHost, b->stream), "read");
  BT_CUDA(b, cudaStreamSynchronize(b->stream), "sync");
  int st = 0;
  BT_CUDA(b, cudaMemcpy(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost), "status");
  if (norm) *norm = out[0];
  if (dipole) *dipole = out[1];
  if (yield) *yield = out[2];
  if (p_ground) *p_ground = out[3];
  if (l_pop) std::memcpy(l_pop, out.data() + 4, sizeof(double) * (I.L + 1));
  if ((st & kStatusNonFinite) || !std::isfinite(out[0]))
    return bfail(b, TDSE_ERR_NONFINITE, "an instance holds Inf/NaN");
  return TDSE_OK;
}

long long tdse_batch_points(const tdse_batch_t *b) { return b ? b->npts : 0; }
long long tdse_batch_launch_count(const tdse_batch_t *b) { return b ? b->launches : 0; }

int tdse_batch_profile(tdse_batch_t *b, int enable) {
  if (!b) return TDSE_ERR_ARG;
  if (b->poisoned) return TDSE_ERR_STATE;
  if (b->profiling) {
    const int rc = bprof_collect(b);
    if (rc) return rc;
  }
  if (enable)
    for (int k = 0; k < TDSE_K_COUNT; ++k) {
      b->prof_ms[k] = 0.0;
      b->prof_n[k] = 0;
    }
  b->profiling = enable != 0;
  return TDSE_OK;
}

int tdse_batch_profile_read(tdse_batch_t *b, int kind, double *total_ms, long long *launches) {
  if (!b) return TDSE_ERR_ARG;
  if (b->poisoned) return TDSE_ERR_STATE;
  if (kind < 0 || kind >= TDSE_K_COUNT) return bfail(b, TDSE_ERR_ARG, "unknown kernel kind");
  if (b->profiling) {
    const int rc = bprof_collect(b);
    if (rc) return rc;
  }
  if (total_ms) *total_ms = b->prof_ms[kind];
  if (launches) *launches = b->prof_n[kind];
  return TDSE_OK;
}

}  // extern "C"
