// Mixed-precision kernels (FP32 stencil arithmetic, FP64 state, dots and norms).
//
// The state psi stays complex128 and every update of psi is done in FP64.  The
// Hamiltonian of Eq. (h_matrix) (arXiv 1308.1856, Sec. 2) is applied in FP32 to
// an operand x = hi + lo + s w, where (hi, lo) is the split of psi into two
// complex64 parts (hi = fl32(psi), lo = fl32(psi - hi), together ~48 bits) and
// w an FP32 work vector (a Krylov vector, a Taylor correction or an RK slope).
//
// Rounding psi itself to FP32 in front of the Laplacian would inject noise of
// ~6e-8 |psi| that the 1/dr^2 stencil amplifies ~600-fold.  Instead the radial
// second derivative is evaluated in difference form: since c0 = -2 c1 - 2 c2,
//   c0 x_j + c1 (x_{j-1} + x_{j+1}) + c2 (x_{j-2} + x_{j+2})
//     = c1 (d_{-1} + d_{+1}) + c2 (d_{-2} + d_{+2}),   d_s = x_{j+s} - x_j,
// and each difference is formed part by part, (hi - hi) + (lo - lo) + s (w - w),
// so its error is relative to the difference, not to psi.  The diagonal table
// then holds l(l+1)/(2 r^2) + V(r) without c0.
//
// In the velocity gauge (VG) the coupling is the (A/c) p_z of the FP64 walker,
// with the first derivatives of rows l - 1 and l + 1 formed in FP32 from
// part-by-part differences as well.
//
// Work decomposition and reductions are those of the FP64 kernels (persistent
// grid, balanced 32-point row segments per warp, fixed-order block partials).
// Each thread sums its FP32 products in an error-free FP32 pair (about twice
// the FP32 precision, no FP64 instruction per point); the block and grid
// reductions of alpha, beta and the norm are FP64.
#include <cuda_runtime.h>

#include <type_traits>

#include "tdse_device_common.cuh"
#include "tdse_stencil.cuh"
#include "tdse_internal.cuh"

namespace tdse_dev {

namespace {

using namespace common;
using namespace stencil;

// Walk this warp's row segments; f(i, idx, Hx, x_center) per point.
// VG: the velocity-gauge coupling.
template <int ST, bool S, bool Wp, bool VG, typename F>
__device__ __forceinline__ void mixed_segments(const MixedIn &in, F &&f) {
  const int lane = threadIdx.x & 31;
  const int N = in.N, Lp1 = in.L + 1;
  const long long NJ = (N + 31) >> 5;
  long long s, s_end;
  warp_range(NJ * Lp1, s, s_end);
  while (s < s_end) {
    const int jg = (int)((unsigned)s / (unsigned)Lp1);
    const int l0 = (int)(s - (long long)jg * Lp1);
    const long long left = s_end - s;
    const int l1 = (left < (long long)(Lp1 - l0)) ? l0 + (int)left : Lp1;
    const int i = jg * 32 + lane;
    if (i < N) mixed_walk_rows<ST, S, Wp, kPrefetchRows, VG>(in, i, l0, l1, f);
    s += l1 - l0;
  }
}

// ---------------------------------------------------------------------------
// psi -> (hi, lo) and the Lanczos start scalars (||psi|| from FP32 products
// summed per thread in an FP32 pair, then across threads in FP64).

__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    mx_split_kernel(size_t G, const double2 *__restrict__ psi, float2 *__restrict__ hi,
                    float2 *__restrict__ lo, Reduction *red, LanczosScalars *ls, int *status) {
  __shared__ double sh[kElemThreads / 32 + 1];
  pdl_wait();
  const int lane = threadIdx.x & 31;
  long long g0, g1;
  warp_range((long long)((G + 31) >> 5), g0, g1);
  PairSum acc;
#pragma unroll 4
  for (long long gi = g0; gi < g1; ++gi) {
    const size_t idx = (size_t)gi * 32 + lane;
    if (idx < G) {
      float2 h, l;
      split2(psi[idx], h, l);
      hi[idx] = h;
      lo[idx] = l;
      acc.add(fmaf(h.x, h.x, h.y * h.y));
    }
  }
  pdl_trigger();
  const double accd = acc.value();
  if (publish_block_partial(accd, red, sh)) {
    const double s = reduce_partials(red, gridDim.x, sh);
    if (threadIdx.x == 0) {
      red->normsq = s;
      const double nrm = sqrt(s);
      ls->psinorm = nrm;
      ls->sigma[0] = (nrm > 0.0) ? 1.0 / nrm : 0.0;
      if (!isfinite(s)) atomicOr(status, kStatusNonFinite);
    }
  }
}

// psi -> (hi, lo) without the norm (operand of the stand-alone mixed H apply).
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    mx_split_plain_kernel(size_t G, const double2 *__restrict__ x, float2 *__restrict__ hi,
                          float2 *__restrict__ lo) {
  const int lane = threadIdx.x & 31;
  long long g0, g1;
  warp_range((long long)((G + 31) >> 5), g0, g1);
#pragma unroll 4
  for (long long gi = g0; gi < g1; ++gi) {
    const size_t idx = (size_t)gi * 32 + lane;
    if (idx < G) {
      float2 h, l;
      split2(x[idx], h, l);
      hi[idx] = h;
      lo[idx] = l;
    }
  }
}

// y = H(E) x in the mixed arithmetic (FP32 stencil on the split of x).
template <int ST, bool VG>
__global__ void __launch_bounds__(kBlockJ, kStencilBlocksPerSM) mx_apply_h_kernel(MixedIn in, double2 *__restrict__ y) {
  mixed_segments<ST, true, false, VG>(in, [&](int, size_t idx, float2 t, float2) {
    y[idx] = make_double2((double)t.x, (double)t.y);
  });
}

// Lanczos iteration j, first half (mixed):
//   z = sigma_j H U_j - (sigma_{j-1} / sigma_j) U_{j-1},  alpha_j = sigma_j Re<U_j, z>,
// with U_0 = psi given as (hi, lo) and U_j (j >= 1) complex64.
template <int ST, bool FIRST, bool VG>
__global__ void __launch_bounds__(kBlockJ, kStencilBlocksPerSM)
    mx_lanczos_a_kernel(MixedIn in, int j, const float2 *__restrict__ uprev,
                        const float2 *__restrict__ prev_hi, const float2 *__restrict__ prev_lo,
                        float2 *__restrict__ z, Reduction *red, LanczosScalars *ls) {
  __shared__ double sh[kBlockJ / 32 + 1];
  pdl_wait();
  const double sigd = ls->sigma[j];
  const float sig = (float)sigd;
  const float cprev = (j > 0) ? (float)ls->ratio[j] : 0.f;
  PairSum acc;
  mixed_segments<ST, FIRST, !FIRST, VG>(in, [&](int, size_t idx, float2 t, float2 u) {
    float2 o = make_float2(sig * t.x, sig * t.y);
    if (!FIRST) {
      float2 up;
      if (uprev) {
        up = uprev[idx];
      } else {   // U_0 = psi
        const float2 h = prev_hi[idx], l = prev_lo[idx];
        up = make_float2(h.x + l.x, h.y + l.y);
      }
      o.x = fmaf(-cprev, up.x, o.x);
      o.y = fmaf(-cprev, up.y, o.y);
    }
    z[idx] = o;
    acc.add(fmaf(u.x, o.x, u.y * o.y));
  });
  pdl_trigger();
  const double accd = acc.value();
  if (publish_block_partial(accd, red, sh)) {
    const double s = reduce_partials(red, gridDim.x, sh);
    if (threadIdx.x == 0) {
      ls->alpha[j] = s * sigd;
      ls->acoef[j] = -(s * sigd) * sigd;
    }
  }
}

// Lanczos iteration j, second half (mixed): U_{j+1} = z - alpha_j sigma_j U_j;
// beta_j = ||U_{j+1}|| (FP32 products, FP32-pair sums, FP64 reduction).
// SPLIT: U_j is U_0 = psi, read as its split (j = 0).
template <bool SPLIT>
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    mx_lanczos_b_kernel(size_t G, int j, const float2 *__restrict__ z, const float2 *__restrict__ u,
                        const float2 *__restrict__ u_hi, const float2 *__restrict__ u_lo,
                        float2 *__restrict__ unext, Reduction *red, LanczosScalars *ls) {
  __shared__ double sh[kElemThreads / 32 + 1];
  pdl_wait();
  const float c = (float)ls->acoef[j];
  const int lane = threadIdx.x & 31;
  long long g0, g1;
  warp_range((long long)((G + 31) >> 5), g0, g1);
  PairSum acc;
#pragma unroll 4
  for (long long gi = g0; gi < g1; ++gi) {
    const size_t idx = (size_t)gi * 32 + lane;
    if (idx < G) {
      float2 uu;
      if (!SPLIT) {
        uu = u[idx];
      } else {
        const float2 h = u_hi[idx], l = u_lo[idx];
        uu = make_float2(h.x + l.x, h.y + l.y);
      }
      const float2 zz = z[idx];
      const float2 o = make_float2(fmaf(c, uu.x, zz.x), fmaf(c, uu.y, zz.y));
      unext[idx] = o;
      acc.add(fmaf(o.x, o.x, o.y * o.y));
    }
  }
  pdl_trigger();
  const double accd = acc.value();
  if (publish_block_partial(accd, red, sh)) {
    const double s = reduce_partials(red, gridDim.x, sh);
    if (threadIdx.x == 0) {
      const double beta = sqrt(s);
      ls->beta[j] = beta;
      const double sn = (beta > 0.0) ? 1.0 / beta : 0.0;
      ls->sigma[j + 1] = sn;
      ls->ratio[j + 1] = (sn > 0.0) ? ls->sigma[j] * beta : 0.0;
    }
  }
}

// psi_new = coef_0 psi + sum_{j>=1} coef_j U_j: the psi term in FP64, the
// Krylov correction summed in FP32 and added in FP64; then the absorber mask,
// the split of psi_new and ||psi_new|| for the next step.
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    mx_lanczos_combine_kernel(size_t G, int N, double2 *psi, float2 *__restrict__ hi,
                              float2 *__restrict__ lo, const float2 *__restrict__ work,
                              size_t stride, const double *__restrict__ mask, int mask_start,
                              Reduction *red, LanczosScalars *ls, int *status) {
  __shared__ double sh[kElemThreads / 32 + 1];
  __shared__ float2 coef[kMaxKrylov];
  __shared__ double2 coef0;
  __shared__ int s_k;
  pdl_wait();
  if (threadIdx.x < kMaxKrylov) {
    const double2 c = ls->coef[threadIdx.x];
    coef[threadIdx.x] = make_float2((float)c.x, (float)c.y);
  }
  if (threadIdx.x == 0) {
    s_k = ls->kdim;
    coef0 = ls->coef[0];
  }
  __syncthreads();
  const int k = s_k;
  const double2 c0 = coef0;
  const int lane = threadIdx.x & 31;
  long long g0, g1;
  warp_range((long long)((G + 31) >> 5), g0, g1);
  PairSum acc;
#pragma unroll 4
  for (long long gi = g0; gi < g1; ++gi) {
    const size_t idx = (size_t)gi * 32 + lane;
    if (idx < G) {
      float cx = 0.f, cy = 0.f;
      for (int jj = 1; jj < k; ++jj) {
        const float2 u = work[(size_t)(jj - 1) * stride + idx];
        const float2 c = coef[jj];
        cx = fmaf(c.x, u.x, cx);
        cx = fmaf(-c.y, u.y, cx);
        cy = fmaf(c.x, u.y, cy);
        cy = fmaf(c.y, u.x, cy);
      }
      const double2 p = psi[idx];
      double ox = fma(c0.x, p.x, fma(-c0.y, p.y, (double)cx));
      double oy = fma(c0.x, p.y, fma(c0.y, p.x, (double)cy));
      const int jr = (int)((unsigned)idx % (unsigned)N);
      if (jr >= mask_start) {
        const double mv = mask[jr];
        ox *= mv;
        oy *= mv;
      }
      const double2 o = make_double2(ox, oy);
      psi[idx] = o;
      float2 h, l;
      split2(o, h, l);
      hi[idx] = h;
      lo[idx] = l;
      acc.add(fmaf(h.x, h.x, h.y * h.y));
    }
  }
  pdl_trigger();
  const double accd = acc.value();
  if (publish_block_partial(accd, red, sh)) {
    const double s = reduce_partials(red, gridDim.x, sh);
    if (threadIdx.x == 0) {
      red->normsq = s;
      const double nrm = sqrt(s);
      ls->psinorm = nrm;
      ls->sigma[0] = (nrm > 0.0) ? 1.0 / nrm : 0.0;
      if (!isfinite(s)) atomicOr(status, kStatusNonFinite);
    }
  }
}

// Taylor stage k in correction form (Horner, Eq. (Taylor)):
//   w_k = (-i dt/k) H (psi + w_{k+1}),  w_{P+1} = 0,  psi_new = psi + w_1.
// The last stage adds w_1 to psi in FP64, applies the mask and re-splits psi.
template <int ST, bool HAS_W, bool VG>
__global__ void __launch_bounds__(kBlockJ, kStencilBlocksPerSM)
    mx_taylor_stage_kernel(MixedIn in, float s, float2 *__restrict__ w_out, int final_stage,
                           double2 *psi, float2 *hi_out, float2 *lo_out,
                           const double *__restrict__ mask, int mask_start) {
  pdl_wait();
  mixed_segments<ST, true, HAS_W, VG>(in, [&](int i, size_t idx, float2 t, float2) {
    const float2 w = make_float2(s * t.y, -s * t.x);   // (-i s)(tx + i ty)
    if (!final_stage) {
      w_out[idx] = w;
    } else {
      const double2 p = psi[idx];
      double ox = p.x + (double)w.x, oy = p.y + (double)w.y;
      if (i >= mask_start) {
        const double mv = mask[i];
        ox *= mv;
        oy *= mv;
      }
      const double2 o = make_double2(ox, oy);
      psi[idx] = o;
      float2 h, l;
      split2(o, h, l);
      hi_out[idx] = h;
      lo_out[idx] = l;
    }
  });
  pdl_trigger();
}

// RK4 stage `stage` (1..4) with k_s = -i H(t_s)(psi + (dt a_s) k_{s-1}):
// stages 1-3 write k_s and add b_s k_s to the compensated FP32 accumulator
// (acc_hi, acc_lo) by an error-free two-sum; stage 4 forms
// psi_new = psi + dt (acc + b_4 k_4) in FP64, masks and re-splits psi.
template <int ST, bool HAS_K, bool VG>
__global__ void __launch_bounds__(kBlockJ, kStencilBlocksPerSM)
    mx_rk_stage_kernel(MixedIn in, int stage, float b, double dtd, float2 *__restrict__ k_out,
                       float2 *acc_hi, float2 *acc_lo, double2 *psi, float2 *hi_out,
                       float2 *lo_out, const double *__restrict__ mask, int mask_start) {
  pdl_wait();
  mixed_segments<ST, true, HAS_K, VG>(in, [&](int i, size_t idx, float2 t, float2) {
    const float2 kv = make_float2(t.y, -t.x);          // -i H g
    const float2 x = make_float2(b * kv.x, b * kv.y);
    if (stage == 1) {
      k_out[idx] = kv;
      acc_hi[idx] = x;
      acc_lo[idx] = make_float2(0.f, 0.f);
    } else if (stage < 4) {
      k_out[idx] = kv;
      const float2 a = acc_hi[idx];
      float2 e = acc_lo[idx];
      // two-sum: a + x = s + err exactly
      const float sx = a.x + x.x, bx = sx - a.x;
      const float sy = a.y + x.y, by = sy - a.y;
      e.x += (a.x - (sx - bx)) + (x.x - bx);
      e.y += (a.y - (sy - by)) + (x.y - by);
      acc_hi[idx] = make_float2(sx, sy);
      acc_lo[idx] = e;
    } else {
      const float2 a = acc_hi[idx], e = acc_lo[idx];
      const double2 p = psi[idx];
      double ox = fma(dtd, (double)a.x + (double)(e.x + x.x), p.x);
      double oy = fma(dtd, (double)a.y + (double)(e.y + x.y), p.y);
      if (i >= mask_start) {
        const double mv = mask[i];
        ox *= mv;
        oy *= mv;
      }
      const double2 o = make_double2(ox, oy);
      psi[idx] = o;
      float2 h, l;
      split2(o, h, l);
      hi_out[idx] = h;
      lo_out[idx] = l;
    }
  });
  pdl_trigger();
}

MixedIn make_mixed(const Geometry &g, const MixedView &mv, float E, const float2 *hi,
                   const float2 *lo, const float2 *w, float ws) {
  MixedIn in;
  in.hi = hi;
  in.lo = lo;
  in.w = w;
  in.ws = ws;
  in.diag = mv.diag;
  in.rj = mv.rj;
  in.kappa = mv.kappa;
  in.pf0 = nullptr;
  in.pf1 = nullptr;
  in.N = g.N;
  in.L = g.L;
  in.c1 = (float)g.c1;
  in.c2 = (float)g.c2;
  in.E = E;
  in.rinv = mv.rinv;
  in.d1c = (float)((g.stencil == 5) ? 1.0 / (12.0 * g.dr) : 1.0 / (2.0 * g.dr));
  return in;
}

template <bool V>
using BC = std::integral_constant<bool, V>;

// f(stencil, velocity gauge) with both as compile-time constants.
template <typename F>
void dispatch(const Geometry &g, F &&f) {
  const bool vg = g.gauge == 1;
  if (g.stencil == 5) {
    if (vg) f(std::integral_constant<int, 5>{}, BC<true>{});
    else f(std::integral_constant<int, 5>{}, BC<false>{});
  } else {
    if (vg) f(std::integral_constant<int, 3>{}, BC<true>{});
    else f(std::integral_constant<int, 3>{}, BC<false>{});
  }
}

inline unsigned stencil_blocks(const Geometry &g) { return (unsigned)(g.sms * kStencilBlocksPerSM); }
inline unsigned elem_blocks(const Geometry &g) { return (unsigned)(g.sms * kElemBlocksPerSM); }

}  // namespace

// ---------------------------------------------------------------------------
cudaError_t launch_mx_split(const Geometry &g, const double2 *psi, float2 *hi, float2 *lo,
                            Reduction *red, LanczosScalars *ls, int *status, cudaStream_t st) {
  const size_t G = (size_t)g.N * (g.L + 1);
  const cudaError_t e = launch_pdl(mx_split_kernel, elem_blocks(g), kElemThreads, 0, st, G, psi, hi, lo, red, ls, status);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_mx_split_plain(const Geometry &g, const double2 *psi, float2 *hi, float2 *lo, cudaStream_t st) {
  const size_t G = (size_t)g.N * (g.L + 1);
  mx_split_plain_kernel<<<elem_blocks(g), kElemThreads, 0, st>>>(G, psi, hi, lo);
  return cudaGetLastError();
}

cudaError_t launch_mx_apply_h(const Geometry &g, const MixedView &mv, double E, const double2 *x,
                              float2 *tmp_hi, float2 *tmp_lo, double2 *y, cudaStream_t st) {
  const size_t G = (size_t)g.N * (g.L + 1);
  mx_split_plain_kernel<<<elem_blocks(g), kElemThreads, 0, st>>>(G, x, tmp_hi, tmp_lo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const MixedIn in = make_mixed(g, mv, (float)E, tmp_hi, tmp_lo, nullptr, 0.f);
  dispatch(g, [&](auto stc, auto vg) {
    mx_apply_h_kernel<decltype(stc)::value, decltype(vg)::value><<<stencil_blocks(g), kBlockJ, 0, st>>>(in, y);
  });
  return cudaGetLastError();
}

cudaError_t launch_mx_lanczos_a(const Geometry &g, const MixedView &mv, double E, int j,
                                const float2 *hi, const float2 *lo, const float2 *u,
                                const float2 *uprev, float2 *z, Reduction *red,
                                LanczosScalars *ls, cudaStream_t st) {
  const unsigned grid = stencil_blocks(g);
  cudaError_t e = cudaSuccess;
  if (j == 0) {
    const MixedIn in = make_mixed(g, mv, (float)E, hi, lo, nullptr, 0.f);
    dispatch(g, [&](auto stc, auto vg) {
      e = launch_pdl(mx_lanczos_a_kernel<decltype(stc)::value, true, decltype(vg)::value>, grid, kBlockJ, 0, st, in, j,
                     nullptr, nullptr, nullptr, z, red, ls);
    });
  } else {
    MixedIn in = make_mixed(g, mv, (float)E, nullptr, nullptr, u, 1.f);
    if (uprev) {
      in.pf0 = uprev;
    } else {
      in.pf0 = hi;
      in.pf1 = lo;
    }
    dispatch(g, [&](auto stc, auto vg) {
      e = launch_pdl(mx_lanczos_a_kernel<decltype(stc)::value, false, decltype(vg)::value>, grid, kBlockJ, 0, st, in, j,
                     uprev, hi, lo, z, red, ls);
    });
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_mx_lanczos_b(const Geometry &g, int j, const float2 *z, const float2 *u,
                                const float2 *hi, const float2 *lo, float2 *unext,
                                Reduction *red, LanczosScalars *ls, cudaStream_t st) {
  const size_t G = (size_t)g.N * (g.L + 1);
  const cudaError_t e =
      u ? launch_pdl(mx_lanczos_b_kernel<false>, elem_blocks(g), kElemThreads, 0, st, G, j, z, u, hi, lo, unext, red, ls)
        : launch_pdl(mx_lanczos_b_kernel<true>, elem_blocks(g), kElemThreads, 0, st, G, j, z, u, hi, lo, unext, red, ls);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_mx_lanczos_combine(const Geometry &g, const OperatorView &op, double2 *psi,
                                      float2 *hi, float2 *lo, const float2 *u1, size_t stride,
                                      Reduction *red, LanczosScalars *ls, int *status,
                                      cudaStream_t st) {
  const size_t G = (size_t)g.N * (g.L + 1);
  const cudaError_t e = launch_pdl(mx_lanczos_combine_kernel, elem_blocks(g), kElemThreads, 0, st, G, g.N, psi, hi, lo,
                                   u1, stride, op.mask, op.mask_start, red, ls, status);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_mx_taylor_stage(const Geometry &g, const MixedView &mv, const OperatorView &op,
                                   double E, double s, const float2 *hi, const float2 *lo,
                                   const float2 *w_in, float2 *w_out, bool final_stage,
                                   double2 *psi, float2 *hi_out, float2 *lo_out, cudaStream_t st) {
  const unsigned grid = stencil_blocks(g);
  const MixedIn in = make_mixed(g, mv, (float)E, hi, lo, w_in, 1.f);
  const int mstart = final_stage ? op.mask_start : g.N;
  const int fs = final_stage ? 1 : 0;
  cudaError_t e = cudaSuccess;
  dispatch(g, [&](auto stc, auto vg) {
    constexpr int ST = decltype(stc)::value;
    constexpr bool VG = decltype(vg)::value;
    if (w_in)
      e = launch_pdl(mx_taylor_stage_kernel<ST, true, VG>, grid, kBlockJ, 0, st, in, (float)s, w_out, fs, psi, hi_out,
                     lo_out, op.mask, mstart);
    else
      e = launch_pdl(mx_taylor_stage_kernel<ST, false, VG>, grid, kBlockJ, 0, st, in, (float)s, w_out, fs, psi, hi_out,
                     lo_out, op.mask, mstart);
  });
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_mx_rk_stage(const Geometry &g, const MixedView &mv, const OperatorView &op,
                               double E, int stage, double dt, const float2 *hi, const float2 *lo,
                               const float2 *k_in, float2 *k_out, float2 *acc_hi, float2 *acc_lo,
                               double2 *psi, float2 *hi_out, float2 *lo_out, cudaStream_t st) {
  // classic tableau: a_{s,s-1} = (-, 1/2, 1/2, 1), b = (1, 2, 2, 1) / 6
  static const float a_in[4] = {0.f, 0.5f, 0.5f, 1.f};
  static const float b[4] = {1.f / 6.f, 1.f / 3.f, 1.f / 3.f, 1.f / 6.f};
  const unsigned grid = stencil_blocks(g);
  const MixedIn in = make_mixed(g, mv, (float)E, hi, lo, k_in, (float)(dt * a_in[stage - 1]));
  const int mstart = (stage == 4) ? op.mask_start : g.N;
  cudaError_t e = cudaSuccess;
  dispatch(g, [&](auto stc, auto vg) {
    constexpr int ST = decltype(stc)::value;
    constexpr bool VG = decltype(vg)::value;
    if (k_in)
      e = launch_pdl(mx_rk_stage_kernel<ST, true, VG>, grid, kBlockJ, 0, st, in, stage, b[stage - 1], dt, k_out, acc_hi,
                     acc_lo, psi, hi_out, lo_out, op.mask, mstart);
    else
      e = launch_pdl(mx_rk_stage_kernel<ST, false, VG>, grid, kBlockJ, 0, st, in, stage, b[stage - 1], dt, k_out, acc_hi,
                     acc_lo, psi, hi_out, lo_out, op.mask, mstart);
  });
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace tdse_dev
