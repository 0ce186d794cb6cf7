// FP64 kernels of the finite-difference TDSE path (sm_103a).
//
// Every stencil kernel evaluates the length-gauge Hamiltonian of Eq. (h_matrix)
// (arXiv 1308.1856, Sec. 2):
//   (H x)_{l,j} = D_{l,j} x_{l,j} + c1 (x_{l,j-1} + x_{l,j+1}) [+ c2 (x_{l,j-2} + x_{l,j+2})]
//               + E r_j (kappa_l x_{l-1,j} + kappa_{l+1} x_{l+1,j})
// with D_{l,j} = c0 + l(l+1)/(2 r_j^2) + V(r_j) read from a table, H real and
// symmetric, so the real and imaginary parts go through the same real operator.
//
// Work decomposition: the grid is persistent (a few blocks per SM) and the
// (L+1) x N points are cut into segments of 32 consecutive radial points of
// one partial wave, ordered radial-group-major.  Warp w takes a contiguous,
// balanced range of the T segments (warp_range), so every warp gets the same
// amount of work to within one segment and the assignment (hence every
// reduction order) is fixed.  Inside a range a lane owns one radial index j
// and walks l upwards keeping x_{l-1,j}, x_{l,j}, x_{l+1,j} in registers, so
// each l-neighbour is loaded once and the coupling coefficient
// kappa_{l+1} E r_j is shared by rows l and l+1.  The radial neighbours come
// from L1/L2 (neighbouring lanes load the same lines).
//
// On GB300 an FP64 instruction issues at 2 lanes/clock/SM, so these kernels
// are FP64-issue bound: the arithmetic is written with explicit __dmul_rn /
// __dadd_rn / __fma_rn so that each grid point costs a known number of FP64
// instructions (5-point Taylor stage: 17).
#include <cuda_runtime.h>

#include <type_traits>

#include "tdse_device_common.cuh"
#include "tdse_stencil.cuh"
#include "tdse_internal.cuh"

namespace tdse_dev {

namespace {

using namespace common;
using namespace stencil;

// Visit this warp's share of the 32-point row segments (see the file header).
template <int ST, bool SCALED = false, bool VG = false, typename F>
__device__ __forceinline__ void for_my_segments(const StencilIn &in, F &&f) {
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
    if (i < in.N) walk_rows<ST, 0, SCALED, VG>(in, i, l0, l1, f);
    s += l1 - l0;
  }
}

// ---------------------------------------------------------------------------
// y = H(E) x
template <int ST, bool VG>
__global__ void __launch_bounds__(kBlockJ, kStencilBlocksPerSM) apply_h_kernel(StencilIn in, double2 *__restrict__ y) {
  for_my_segments<ST, false, VG>(in, [&](int, size_t idx, double2 t, double2) { y[idx] = t; });
}

// Horner stage of the Taylor polynomial (Eq. (Taylor)):
//   v_out = psi + (-i s) H v_in,  s = dt / k   (IMAG: psi - s H v_in, Sec. 3's
//   imaginary-time propagation).
// The last stage (k = 1, FIN) writes psi itself and applies the absorber
// mask; the other stages carry no mask code at all (a predicated-off FP64
// instruction still takes its issue slot on the FP64 pipe).
template <int ST, bool IMAG, bool VG, bool FIN>
__global__ void __launch_bounds__(kBlockJ, kStencilBlocksPerSM)
    taylor_stage_kernel(StencilIn in, double s, const double2 *__restrict__ psi,
                        double2 *__restrict__ out, const double *__restrict__ mask,
                        int mask_start) {
  pdl_wait();
  for_my_segments<ST, false, VG>(in, [&](int i, size_t idx, double2 t, double2) {
    const bool masked = FIN && i >= mask_start;
    const double2 p = psi[idx];
    double2 o;
    if (IMAG) {
      o.x = __fma_rn(-s, t.x, p.x);
      o.y = __fma_rn(-s, t.y, p.y);
    } else {
      o.x = __fma_rn(s, t.y, p.x);     // (-i s)(tx + i ty) = s ty - i s tx
      o.y = __fma_rn(-s, t.x, p.y);
    }
    if (masked) { const double mv = mask[i]; o.x = __dmul_rn(mv, o.x); o.y = __dmul_rn(mv, o.y); }
    out[idx] = o;
  });
  pdl_trigger();
}

// Stage `stage` (1..4) of classic RK4 (Eq. (RKDeriv)) with k = -i H(t_n + c dt) g:
//   stages 1-3: g_next = psi + (dt a) k,  acc_out = acc_in + (dt b) k  (acc_in = psi at stage 1)
//   stage 4:    psi    = acc_in + (dt b) k, then the absorber mask.
// IMAG: k = -H g (imaginary time) instead of -i H g.
template <int ST, bool IMAG, bool VG>
__global__ void __launch_bounds__(kBlockJ, kStencilBlocksPerSM)
    rk_stage_kernel(StencilIn in, int stage, double ca, double cb,
                    const double2 *__restrict__ psi, const double2 *__restrict__ acc_in,
                    double2 *__restrict__ acc_out, double2 *__restrict__ g_next,
                    double2 *__restrict__ psi_out, const double *__restrict__ mask,
                    int mask_start) {
  const int mstart = (stage == 4) ? mask_start : in.N;
  pdl_wait();
  for_my_segments<ST, false, VG>(in, [&](int i, size_t idx, double2 t, double2) {
    const double2 a = acc_in[idx];
    // c k with k = -i t:  (c t.y, -c t.x);  with k = -t:  (-c t.x, -c t.y)
    auto add = [&](double c, double2 base) {
      return IMAG ? make_double2(__fma_rn(-c, t.x, base.x), __fma_rn(-c, t.y, base.y))
                  : make_double2(__fma_rn(c, t.y, base.x), __fma_rn(-c, t.x, base.y));
    };
    if (stage < 4) {
      const double2 p = psi[idx];
      g_next[idx] = add(ca, p);
      acc_out[idx] = add(cb, a);
    } else {
      double2 o = add(cb, a);
      if (i >= mstart) { const double mv = mask[i]; o.x = __dmul_rn(mv, o.x); o.y = __dmul_rn(mv, o.y); }
      psi_out[idx] = o;
    }
  });
  pdl_trigger();
}

// Stage a.stage of a general explicit Runge-Kutta method (appendix
// "Runge-Kutta"); see RkStageArgs.  NK = a.stage + 1 terms and MODE are
// compile-time, so no FP64 instruction is issued for absent terms (a
// predicated-off FP64 instruction still takes its FP64 issue slot):
//   MODE 0: an inner stage (k_i and g_{i+1} out);
//   MODE 1: the last stage (psi, Delta and the sigma partial);
//   MODE 2: the last stage of a first-same-as-last tableau (b_{s-1} = 0 and
//           a_{s-1,j} = b_j): psi_new is the stage's own input g_{s-1}, which
//           the previous stage summed in the same order with the same
//           coefficients, so only Delta is formed.
// The slopes of the earlier stages are read pointwise and combined in stage
// order, the new slope k_i = -i H g_i last, so the sums round in the same
// order as the oracle's.
template <int ST, bool VG, int NK, int MODE>
__global__ void __launch_bounds__(kBlockJ, kStencilBlocksPerSM)
    rk_general_stage_kernel(StencilIn in, RkStageArgs a, const double2 *__restrict__ psi,
                            const double *__restrict__ mask, int mask_start, Reduction *red,
                            double S) {
  constexpr bool LAST = MODE != 0;
  constexpr bool FSAL = MODE == 2;
  __shared__ double sh[kBlockJ / 32 + 1];
  double acc = 0.0;
  pdl_wait();
  for_my_segments<ST, false, VG>(in, [&](int r, size_t idx, double2 t, double2 u) {
    const double2 ki = make_double2(t.y, -t.x);   // -i (tx + i ty)
    double2 kj[NK > 1 ? NK - 1 : 1];
#pragma unroll
    for (int j = 0; j < NK - 1; ++j) kj[j] = a.k[j][idx];
    double2 o = FSAL ? u : psi[idx];
    double2 d = make_double2(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < NK - 1; ++j) {
      if (!FSAL) {
        o.x = __fma_rn(a.coef[j], kj[j].x, o.x);
        o.y = __fma_rn(a.coef[j], kj[j].y, o.y);
      }
      if (LAST) {
        d.x = __fma_rn(a.dcoef[j], kj[j].x, d.x);
        d.y = __fma_rn(a.dcoef[j], kj[j].y, d.y);
      }
    }
    if (!FSAL) {
      o.x = __fma_rn(a.coef[NK - 1], ki.x, o.x);
      o.y = __fma_rn(a.coef[NK - 1], ki.y, o.y);
    }
    if (!LAST) {
      a.k_out[idx] = ki;
      a.g_out[idx] = o;
    } else {
      d.x = __fma_rn(a.dcoef[NK - 1], ki.x, d.x);
      d.y = __fma_rn(a.dcoef[NK - 1], ki.y, d.y);
      acc = __fma_rn(d.x, d.x, acc);
      acc = __fma_rn(d.y, d.y, acc);
      if (r >= mask_start) { const double mv = mask[r]; o.x = __dmul_rn(mv, o.x); o.y = __dmul_rn(mv, o.y); }
      a.psi_out[idx] = o;
    }
  });
  pdl_trigger();
  if (LAST && publish_block_partial(acc, red, sh)) {
    const double s = reduce_partials(red, gridDim.x, sh);
    if (threadIdx.x == 0) {
      *a.sigma += sqrt(s / S);
      if (!isfinite(s)) atomicOr(a.status, kStatusNonFinite);
    }
  }
}

// Lanczos iteration j, first half (Appendix "Lanczos methods"):
//   z = H q_j - beta_{j-1} q_{j-1},   q_j = sigma_j U_j,
//   beta_{j-1} q_{j-1} = (sigma_{j-1} / sigma_j) U_{j-1},
//   alpha_j = Re <q_j, z> = sigma_j Re <U_j, z>  (grid reduction; last block stores it).
template <int ST, bool VG>
__global__ void __launch_bounds__(kBlockJ, kStencilBlocksPerSM)
    lanczos_a_kernel(StencilIn in, int j, const double2 *__restrict__ uprev,
                     double2 *__restrict__ z, Reduction *red, LanczosScalars *ls) {
  __shared__ double sh[kBlockJ / 32 + 1];
  pdl_wait();
  const double sig = ls->sigma[j];
  const double cprev = (j > 0) ? ls->ratio[j] : 0.0;
  double acc = 0.0;
  // t = sigma_j H U_j directly (the operator scaled by sigma_j)
  for_my_segments<ST, true, VG>(scaled(in, sig), [&](int, size_t idx, double2 t, double2 u) {
    double2 o;
    if (j > 0) {
      const double2 up = uprev[idx];
      o.x = __fma_rn(-cprev, up.x, t.x);
      o.y = __fma_rn(-cprev, up.y, t.y);
    } else {
      o = t;
    }
    z[idx] = o;
    acc = __fma_rn(u.x, o.x, acc);
    acc = __fma_rn(u.y, o.y, acc);
  });
  pdl_trigger();
  if (publish_block_partial(acc, red, sh)) {
    const double s = reduce_partials(red, gridDim.x, sh);
    if (threadIdx.x == 0) {
      ls->alpha[j] = s * sig;
      ls->acoef[j] = -(s * sig) * sig;
    }
  }
}

// Elementwise kernels: persistent grid; each warp takes a contiguous, balanced
// range of the groups of 32 consecutive elements (warp_range).

template <typename F>
__device__ __forceinline__ void for_my_groups(size_t G, F &&f) {
  const int lane = threadIdx.x & 31;
  long long g0, g1;
  warp_range((long long)((G + 31) >> 5), g0, g1);
  for (long long gi = g0; gi < g1; ++gi) {
    const size_t idx = (size_t)gi * 32 + lane;
    if (idx < G) f(idx);
  }
}

// Up to kUnroll groups of this warp's range are loaded before any of them is
// used, so their memory latencies overlap.
constexpr int kUnroll = 4;

// Lanczos iteration j, second half: U_{j+1} = z - alpha_j sigma_j U_j; beta_j = ||U_{j+1}||.
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    lanczos_b_kernel(size_t G, int j, const double2 *__restrict__ z, const double2 *__restrict__ u,
                     double2 *__restrict__ unext, Reduction *red, LanczosScalars *ls) {
  __shared__ double sh[kElemThreads / 32 + 1];
  pdl_wait();
  const double c = ls->acoef[j];
  double acc0 = 0.0, acc1 = 0.0;
  const int lane = threadIdx.x & 31;
  long long g0, g1;
  warp_range((long long)((G + 31) >> 5), g0, g1);
  for (long long gb = g0; gb < g1; gb += kUnroll) {
    double2 zz[kUnroll], uu[kUnroll];
#pragma unroll
    for (int r = 0; r < kUnroll; ++r) {
      const size_t idx = (size_t)(gb + r) * 32 + lane;
      const bool ok = (gb + r < g1) && idx < G;
      zz[r] = ok ? z[idx] : make_double2(0.0, 0.0);
      uu[r] = ok ? u[idx] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int r = 0; r < kUnroll; ++r) {
      const size_t idx = (size_t)(gb + r) * 32 + lane;
      if ((gb + r < g1) && idx < G) {
        const double2 o = make_double2(__fma_rn(c, uu[r].x, zz[r].x), __fma_rn(c, uu[r].y, zz[r].y));
        unext[idx] = o;
        acc0 = __fma_rn(o.x, o.x, acc0);
        acc1 = __fma_rn(o.y, o.y, acc1);
      }
    }
  }
  pdl_trigger();
  if (publish_block_partial(acc0 + acc1, red, sh)) {
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

// ||x||^2 -> Lanczos start scalars (sigma_0 = 1/||psi||, psinorm) and the
// non-finite status bit.
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    norm_kernel(size_t G, const double2 *__restrict__ x, Reduction *red, LanczosScalars *ls,
                int *status) {
  __shared__ double sh[kElemThreads / 32 + 1];
  pdl_wait();
  double acc0 = 0.0, acc1 = 0.0;
  const int lane = threadIdx.x & 31;
  long long g0, g1;
  warp_range((long long)((G + 31) >> 5), g0, g1);
  for (long long gb = g0; gb < g1; gb += kUnroll) {
    double2 v[kUnroll];
#pragma unroll
    for (int r = 0; r < kUnroll; ++r) {
      const size_t idx = (size_t)(gb + r) * 32 + lane;
      v[r] = ((gb + r < g1) && idx < G) ? x[idx] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int r = 0; r < kUnroll; ++r) {
      acc0 = __fma_rn(v[r].x, v[r].x, acc0);
      acc1 = __fma_rn(v[r].y, v[r].y, acc1);
    }
  }
  pdl_trigger();
  if (publish_block_partial(acc0 + acc1, red, sh)) {
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

// Imaginary time (Sec. 3): the squared norm before a step, then after it the
// energy estimate and the renormalisation of psi.
__global__ void imag_begin_kernel(const Reduction *red, double dr, double *imag) {
  imag[0] = dr * red->normsq;
}

__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    imag_normalize_kernel(size_t G, double2 *psi, const Reduction *red, double dr, double dt,
                          double *imag) {
  const double n2 = dr * red->normsq;
  const double sc = (n2 > 0.0) ? 1.0 / sqrt(n2) : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) imag[1] = -log(n2 / imag[0]) / (2.0 * dt);
  for_my_groups(G, [&](size_t idx) {
    const double2 v = psi[idx];
    psi[idx] = make_double2(__dmul_rn(sc, v.x), __dmul_rn(sc, v.y));
  });
}

// psi_new = sum_{j<k} coef_j U_j  (U_0 = psi, read and written in place by
// the same thread), then the absorber mask and ||psi_new||^2 for the next step.
__global__ void __launch_bounds__(kElemThreads, kElemBlocksPerSM)
    lanczos_combine_kernel(size_t G, int N, double2 *psi, const double2 *__restrict__ work,
                           size_t stride, const double *__restrict__ mask, int mask_start,
                           Reduction *red, LanczosScalars *ls, int *status) {
  __shared__ double sh[kElemThreads / 32 + 1];
  __shared__ double2 coef[kMaxKrylov];
  __shared__ int s_k;
  pdl_wait();
  if (threadIdx.x < kMaxKrylov) coef[threadIdx.x] = ls->coef[threadIdx.x];
  if (threadIdx.x == 0) s_k = ls->kdim;
  __syncthreads();
  const int k = s_k;
  double acc = 0.0;
  for_my_groups(G, [&](size_t idx) {
    const double2 u0 = psi[idx];
    double ox = __fma_rn(coef[0].x, u0.x, __dmul_rn(-coef[0].y, u0.y));
    double oy = __fma_rn(coef[0].x, u0.y, __dmul_rn(coef[0].y, u0.x));
    for (int jj = 1; jj < k; ++jj) {
      const double2 u = work[(size_t)(jj - 1) * stride + idx];
      const double2 c = coef[jj];
      ox = __fma_rn(c.x, u.x, ox);
      ox = __fma_rn(-c.y, u.y, ox);
      oy = __fma_rn(c.x, u.y, oy);
      oy = __fma_rn(c.y, u.x, oy);
    }
    const int jr = (int)((unsigned)idx % (unsigned)N);
    if (jr >= mask_start) {
      const double mv = mask[jr];
      ox = __dmul_rn(mv, ox);
      oy = __dmul_rn(mv, oy);
    }
    psi[idx] = make_double2(ox, oy);
    acc = __fma_rn(ox, ox, acc);
    acc = __fma_rn(oy, oy, acc);
  });
  pdl_trigger();
  if (publish_block_partial(acc, red, sh)) {
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

// Observables (Sec. 4): per block of row l, partial sums of
//   q0: sum |f|^2, q1: sum_{r_j <= r_b} |f|^2, q2: sum r_j Re(conj(f_l) f_{l+1}),
//   q3, q4: sum conj(ref_j) f_{0,j} (row 0 only).
// Partials are laid out [q][row][bx]; the last block combines them in index
// order into out = {norm, dipole, yield, p_ground, l_pop[0..L]}.
constexpr int kObsThreads = 256;
constexpr int kObsQ = 5;

__global__ void __launch_bounds__(kObsThreads)
    observables_kernel(const double2 *__restrict__ psi, const double2 *__restrict__ ref0,
                       const double *__restrict__ rj, const double *__restrict__ kappa,
                       int N, int L, double dr, double r_b, double *partials,
                       unsigned *ticket, double *out) {
  __shared__ double sh[kObsThreads / 32 + 1];
  __shared__ unsigned s_last;
  const int l = blockIdx.y;
  const int nbx = gridDim.x;
  double q[kObsQ] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = blockIdx.x * kObsThreads + threadIdx.x; i < N; i += nbx * kObsThreads) {
    const size_t idx = (size_t)l * N + i;
    const double2 f = psi[idx];
    const double a = __fma_rn(f.x, f.x, __dmul_rn(f.y, f.y));
    const double r = rj[i];
    q[0] += a;
    if (r <= r_b) q[1] += a;
    if (l < L) {
      const double2 g = psi[idx + N];
      q[2] = __fma_rn(r, __fma_rn(f.x, g.x, __dmul_rn(f.y, g.y)), q[2]);
    }
    if (l == 0 && ref0) {
      const double2 c = ref0[i];
      q[3] += __fma_rn(c.x, f.x, __dmul_rn(c.y, f.y));    // Re(conj(c) f)
      q[4] += __fma_rn(c.x, f.y, __dmul_rn(-c.y, f.x));   // Im(conj(c) f)
    }
  }
  const size_t nb = (size_t)nbx * (L + 1);
  const size_t bid = (size_t)l * nbx + blockIdx.x;
  for (int k = 0; k < kObsQ; ++k) {
    const double b = block_sum(q[k], sh);
    if (threadIdx.x == 0) partials[(size_t)k * nb + bid] = b;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(ticket, 1u) == nb - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last block: per-row sums in fixed order (thread t handles rows t, t+256, ...)
  double norm_part = 0.0, inside_part = 0.0, dip_part = 0.0;
  for (int row = threadIdx.x; row <= L; row += kObsThreads) {
    double p0 = 0.0, p1 = 0.0, p2 = 0.0;
    for (int bx = 0; bx < nbx; ++bx) {
      const size_t o = (size_t)row * nbx + bx;
      p0 += __ldcg(&partials[0 * nb + o]);
      p1 += __ldcg(&partials[1 * nb + o]);
      p2 += __ldcg(&partials[2 * nb + o]);
    }
    out[4 + row] = dr * p0;
    norm_part += p0;
    inside_part += p1;
    if (row < L) dip_part += 2.0 * kappa[row + 1] * dr * p2;
  }
  const double norm = block_sum(norm_part, sh);
  const double inside = block_sum(inside_part, sh);
  const double dip = block_sum(dip_part, sh);
  if (threadIdx.x == 0) {
    double ore = 0.0, oim = 0.0;
    for (int bx = 0; bx < nbx; ++bx) {
      ore += __ldcg(&partials[3 * nb + bx]);
      oim += __ldcg(&partials[4 * nb + bx]);
    }
    ore *= dr;
    oim *= dr;
    out[0] = dr * norm;
    out[1] = dip;
    out[2] = 1.0 - dr * inside;
    out[3] = ore * ore + oim * oim;
    *ticket = 0u;
  }
}

StencilIn make_in(const Geometry &g, const OperatorView &op, double E, const double2 *x) {
  StencilIn in;
  in.x = x;
  in.diag = op.diag;
  in.rj = op.rj;
  in.kappa = op.kappa;
  in.N = g.N;
  in.L = g.L;
  in.c1 = g.c1;
  in.c2 = g.c2;
  in.E = E;
  in.dscale = 1.0;
  in.rinv = op.rinv;
  in.d1c = (g.stencil == 5) ? 1.0 / (12.0 * g.dr) : 1.0 / (2.0 * g.dr);
  return in;
}

template <int V>
using IC = std::integral_constant<int, V>;
template <bool V>
using BC = std::integral_constant<bool, V>;

// f(stencil, velocity gauge) with both as compile-time constants.
template <typename F>
void dispatch(const Geometry &g, bool vg, F &&f) {
  if (g.stencil == 5) {
    if (vg) f(IC<5>{}, BC<true>{});
    else f(IC<5>{}, BC<false>{});
  } else {
    if (vg) f(IC<3>{}, BC<true>{});
    else f(IC<3>{}, BC<false>{});
  }
}

// Persistent grids: a few blocks per SM (all resident at once).
inline unsigned stencil_blocks(const Geometry &g) { return (unsigned)(g.sms * kStencilBlocksPerSM); }
inline unsigned elem_blocks(const Geometry &g) { return (unsigned)(g.sms * kElemBlocksPerSM); }

}  // namespace

// ---------------------------------------------------------------------------
cudaError_t launch_apply_h(const Geometry &g, const OperatorView &op, double E,
                           const double2 *x, double2 *y, cudaStream_t s) {
  const StencilIn in = make_in(g, op, E, x);
  const unsigned grid = stencil_blocks(g);
  dispatch(g, g.gauge == 1, [&](auto st, auto vg) {
    apply_h_kernel<decltype(st)::value, decltype(vg)::value><<<grid, kBlockJ, 0, s>>>(in, y);
  });
  return cudaGetLastError();
}

cudaError_t launch_taylor_stage(const Geometry &g, const OperatorView &op, double E, double s,
                                const double2 *v_in, const double2 *psi, double2 *v_out,
                                bool final_stage, cudaStream_t st, bool imag) {
  const StencilIn in = make_in(g, op, E, v_in);
  const unsigned grid = stencil_blocks(g);
  const int mstart = op.mask_start;
  cudaError_t e = cudaSuccess;
  dispatch(g, !imag && g.gauge == 1, [&](auto stc, auto vg) {
    constexpr int ST = decltype(stc)::value;
    constexpr bool VG = decltype(vg)::value;
    if (imag)   // imaginary time: no absorber, no field
      e = launch_pdl(taylor_stage_kernel<ST, true, false, false>, grid, kBlockJ, 0, st, in, s, psi, v_out, op.mask, mstart);
    else if (final_stage)
      e = launch_pdl(taylor_stage_kernel<ST, false, VG, true>, grid, kBlockJ, 0, st, in, s, psi, v_out, op.mask, mstart);
    else
      e = launch_pdl(taylor_stage_kernel<ST, false, VG, false>, grid, kBlockJ, 0, st, in, s, psi, v_out, op.mask, mstart);
  });
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_rk_stage(const Geometry &g, const OperatorView &op, double E, int stage,
                            double dt, const double2 *gin, const double2 *psi,
                            const double2 *acc_in, double2 *acc_out, double2 *g_next,
                            double2 *psi_out, cudaStream_t st, bool imag) {
  // classic tableau: a_{s+1,s} = (1/2, 1/2, 1), b = (1, 2, 2, 1) / 6
  static const double a_next[4] = {0.5, 0.5, 1.0, 0.0};
  static const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  const StencilIn in = make_in(g, op, E, gin);
  const unsigned grid = stencil_blocks(g);
  const double ca = dt * a_next[stage - 1], cb = dt * b[stage - 1];
  const int mstart = imag ? g.N : op.mask_start;
  cudaError_t e = cudaSuccess;
  dispatch(g, !imag && g.gauge == 1, [&](auto stc, auto vg) {
    constexpr int ST = decltype(stc)::value;
    constexpr bool VG = decltype(vg)::value;
    if (imag)
      e = launch_pdl(rk_stage_kernel<ST, true, false>, grid, kBlockJ, 0, st, in, stage, ca, cb, psi, acc_in, acc_out,
                     g_next, psi_out, op.mask, mstart);
    else
      e = launch_pdl(rk_stage_kernel<ST, false, VG>, grid, kBlockJ, 0, st, in, stage, ca, cb, psi, acc_in, acc_out,
                     g_next, psi_out, op.mask, mstart);
  });
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_rk_general_stage(const Geometry &g, const OperatorView &op, double E,
                                    const double2 *gin, const double2 *psi, const RkStageArgs &a,
                                    Reduction *red, cudaStream_t st) {
  if (a.stage < 0 || a.stage >= kRkMaxStages) return cudaErrorInvalidValue;
  const StencilIn in = make_in(g, op, E, gin);
  const unsigned grid = stencil_blocks(g);
  const double S = (double)g.N * (double)(g.L + 1);
  const int mode = a.last ? (a.fsal ? 2 : 1) : 0;
  cudaError_t e = cudaSuccess;
  if (!a.last && a.stage == kRkMaxStages - 1) return cudaErrorInvalidValue;   // no stage after the last
  if (a.fsal && (!a.last || a.stage == 0)) return cudaErrorInvalidValue;
  dispatch(g, g.gauge == 1, [&](auto stc, auto vg) {
    constexpr int ST = decltype(stc)::value;
    constexpr bool VG = decltype(vg)::value;
    auto go = [&](auto nk) {
      constexpr int NK = decltype(nk)::value;
      if (mode == 1)
        e = launch_pdl(rk_general_stage_kernel<ST, VG, NK, 1>, grid, kBlockJ, 0, st, in, a, psi, op.mask,
                       op.mask_start, red, S);
      else if constexpr (NK > 1)
        if (mode == 2)
          e = launch_pdl(rk_general_stage_kernel<ST, VG, NK, 2>, grid, kBlockJ, 0, st, in, a, psi, op.mask,
                         op.mask_start, red, S);
      if constexpr (NK < kRkMaxStages)
        if (mode == 0)
          e = launch_pdl(rk_general_stage_kernel<ST, VG, NK, 0>, grid, kBlockJ, 0, st, in, a, psi, op.mask,
                         op.mask_start, red, S);
    };
    switch (a.stage + 1) {
      case 1: go(IC<1>{}); break;
      case 2: go(IC<2>{}); break;
      case 3: go(IC<3>{}); break;
      case 4: go(IC<4>{}); break;
      case 5: go(IC<5>{}); break;
      case 6: go(IC<6>{}); break;
      default: go(IC<7>{}); break;
    }
  });
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_imag_begin(const Reduction *red, double dr, double *imag_dev, cudaStream_t st) {
  imag_begin_kernel<<<1, 1, 0, st>>>(red, dr, imag_dev);
  return cudaGetLastError();
}

cudaError_t launch_imag_normalize(const Geometry &g, double2 *psi, const Reduction *red, double dt,
                                  double *imag_dev, cudaStream_t st) {
  const size_t G = (size_t)g.N * (g.L + 1);
  imag_normalize_kernel<<<elem_blocks(g), kElemThreads, 0, st>>>(G, psi, red, g.dr, dt, imag_dev);
  return cudaGetLastError();
}

cudaError_t launch_norm(const Geometry &g, const double2 *x, Reduction *red,
                        LanczosScalars *ls, int *status, cudaStream_t st) {
  const size_t G = (size_t)g.N * (g.L + 1);
  const cudaError_t e = launch_pdl(norm_kernel, elem_blocks(g), kElemThreads, 0, st, G, x, red, ls, status);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_lanczos_a(const Geometry &g, const OperatorView &op, double E, int j,
                             const double2 *u, const double2 *uprev, double2 *z,
                             Reduction *red, LanczosScalars *ls, cudaStream_t st) {
  const StencilIn in = make_in(g, op, E, u);
  const unsigned grid = stencil_blocks(g);
  cudaError_t e = cudaSuccess;
  dispatch(g, g.gauge == 1, [&](auto stc, auto vg) {
    e = launch_pdl(lanczos_a_kernel<decltype(stc)::value, decltype(vg)::value>, grid, kBlockJ, 0, st, in, j, uprev,
                   z, red, ls);
  });
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_lanczos_b(const Geometry &g, int j, const double2 *z, const double2 *u,
                             double2 *unext, Reduction *red, LanczosScalars *ls, cudaStream_t st) {
  const size_t G = (size_t)g.N * (g.L + 1);
  const cudaError_t e = launch_pdl(lanczos_b_kernel, elem_blocks(g), kElemThreads, 0, st, G, j, z, u, unext, red, ls);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_lanczos_combine(const Geometry &g, const OperatorView &op, int m,
                                   double2 *psi, const double2 *work, size_t stride,
                                   Reduction *red, LanczosScalars *ls, int *status,
                                   cudaStream_t st) {
  (void)m;
  const size_t G = (size_t)g.N * (g.L + 1);
  const cudaError_t e = launch_pdl(lanczos_combine_kernel, elem_blocks(g), kElemThreads, 0, st, G, g.N, psi, work,
                                   stride, op.mask, op.mask_start, red, ls, status);
  return e != cudaSuccess ? e : cudaGetLastError();
}

int observables_blocks(const Geometry &g) {
  const int per_row = (g.N + kObsThreads - 1) / kObsThreads;
  return per_row < 8 ? per_row : 8;
}

cudaError_t launch_observables(const Geometry &g, const OperatorView &op, const double2 *psi,
                               const double2 *ref0, double r_b, double *partials,
                               unsigned *ticket, double *out, cudaStream_t st) {
  const int nbx = observables_blocks(g);
  const dim3 grid(nbx, g.L + 1);
  observables_kernel<<<grid, kObsThreads, 0, st>>>(psi, ref0, op.rj, op.kappa, g.N, g.L, g.dr,
                                                   r_b, partials, ticket, out);
  return cudaGetLastError();
}

}  // namespace tdse_dev
