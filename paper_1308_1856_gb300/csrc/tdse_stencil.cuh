// Point evaluators of the Hamiltonian shared by the single-instance and the
// batched kernels: the FP64 stencil (Sec. 2, Eq. (h_matrix) of arXiv 1308.1856)
// and the mixed-precision operand (FP32 parts, difference-form Laplacian).
#pragma once

#include <cuda_runtime.h>

namespace tdse_dev {
namespace stencil {

__device__ __forceinline__ double2 ldg2(const double2 *p) { return __ldg(p); }
// The operand's load: read-only (non-coherent) path, or CG: from L2, for a
// kernel whose other blocks rewrite the operand between its phases (an SM's
// L1 is not kept coherent with another SM's stores).
template <bool CG>
__device__ __forceinline__ double2 ldx(const double2 *p) { return CG ? __ldcg(p) : __ldg(p); }

// Rows ahead of the current one whose lines the mixed walker asks L2 for.
// The walk visits one row per iteration with little arithmetic, so a load
// issued one row ahead does not cover DRAM latency at the occupancy these
// kernels run at; prefetches (no destination register) go further ahead.
constexpr int kPrefetchRows = 6;

__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}


struct StencilIn {
  const double2 *__restrict__ x;
  const double *__restrict__ diag;
  const double *__restrict__ rj;
  const double *__restrict__ kappa;
  int N, L;
  double c1, c2, E;  // E: the field (length gauge) or A/c (velocity gauge)
  double dscale;   // walkers with SCALED multiply the diagonal by it (the other terms
                   // are scaled through c1, c2 and E by the caller)
  const double *__restrict__ rinv;   // velocity gauge: 1 / r_j
  double d1c;                        // velocity gauge: 1/(12 dr) (5-point) or 1/(2 dr) (3-point)
};

// First derivative of a row at column i (zero beyond the box): Sec. 2's
// 4th-order formula [-f_{j+2} + 8 f_{j+1} - 8 f_{j-1} + f_{j-2}] / (12 dr), or
// [f_{j+1} - f_{j-1}] / (2 dr) with the 3-point stencil.
template <int ST>
__device__ __forceinline__ double2 d1_point(const StencilIn &in, const double2 *row, int i) {
  const double2 z = make_double2(0.0, 0.0);
  const double2 m1 = (i >= 1) ? ldg2(row + i - 1) : z;
  const double2 p1 = (i + 1 < in.N) ? ldg2(row + i + 1) : z;
  if (ST == 5) {
    const double2 m2 = (i >= 2) ? ldg2(row + i - 2) : z;
    const double2 p2 = (i + 2 < in.N) ? ldg2(row + i + 2) : z;
    return make_double2(
        __dmul_rn(in.d1c, __fma_rn(8.0, __dsub_rn(p1.x, m1.x), __dsub_rn(m2.x, p2.x))),
        __dmul_rn(in.d1c, __fma_rn(8.0, __dsub_rn(p1.y, m1.y), __dsub_rn(m2.y, p2.y))));
  }
  return make_double2(__dmul_rn(in.d1c, __dsub_rn(p1.x, m1.x)), __dmul_rn(in.d1c, __dsub_rn(p1.y, m1.y)));
}

// The operator scaled by s: every coefficient that multiplies the operand is
// multiplied by s once (c1, c2, E here, the diagonal point by point by the
// SCALED walker), so s H x costs one FP64 multiply per point instead of two.
__device__ __forceinline__ StencilIn scaled(StencilIn in, double s) {
  in.c1 = __dmul_rn(s, in.c1);
  in.c2 = __dmul_rn(s, in.c2);
  in.E = __dmul_rn(s, in.E);
  in.dscale = s;
  return in;
}

// (H x) at (l, i) from the register window; 15 FP64 instructions (5-point).
// LG = false leaves out the length-gauge coupling (the velocity gauge adds its own).
template <int ST, bool LG = true, bool CG = false>
__device__ __forceinline__ double2 h_point(const StencilIn &in, const double2 *row, int i,
                                           double d, double2 prev, double2 cur, double2 next,
                                           double a_cur, double a_next) {
  const double2 z = make_double2(0.0, 0.0);
  const double2 m1 = (i >= 1) ? ldx<CG>(row + i - 1) : z;
  const double2 p1 = (i + 1 < in.N) ? ldx<CG>(row + i + 1) : z;
  double tx = __dmul_rn(d, cur.x);
  double ty = __dmul_rn(d, cur.y);
  tx = __fma_rn(in.c1, __dadd_rn(m1.x, p1.x), tx);
  ty = __fma_rn(in.c1, __dadd_rn(m1.y, p1.y), ty);
  if (ST == 5) {
    const double2 m2 = (i >= 2) ? ldx<CG>(row + i - 2) : z;
    const double2 p2 = (i + 2 < in.N) ? ldx<CG>(row + i + 2) : z;
    tx = __fma_rn(in.c2, __dadd_rn(m2.x, p2.x), tx);
    ty = __fma_rn(in.c2, __dadd_rn(m2.y, p2.y), ty);
  }
  if (LG) {
    tx = __fma_rn(a_cur, prev.x, tx);
    ty = __fma_rn(a_cur, prev.y, ty);
    tx = __fma_rn(a_next, next.x, tx);
    ty = __fma_rn(a_next, next.y, ty);
  }
  return make_double2(tx, ty);
}

struct MixedIn {
  const float2 *__restrict__ hi;   // split of psi (may be null)
  const float2 *__restrict__ lo;
  const float2 *__restrict__ w;    // FP32 work vector (may be null)
  float ws;                        // scale of w in the operand
  const float *__restrict__ diag;  // l(l+1)/(2 r^2) + V(r) (+ odd-ghost fold), no c0
  const float *__restrict__ rj;
  const float *__restrict__ kappa;
  const float2 *pf0, *pf1;         // rows the caller's epilogue reads at the same index (may be null)
  int N, L;
  float c1, c2, E;                 // E: the field (length gauge) or A/c (velocity gauge)
  const float *__restrict__ rinv;  // velocity gauge: 1 / r_j (else unused)
  float d1c;                       // velocity gauge: 1/(12 dr) (5-point) or 1/(2 dr) (3-point)
};

// L2 prefetch of every array the walker and its epilogue read at row offset idx.
template <bool S, bool Wp>
__device__ __forceinline__ void prefetch_row(const MixedIn &in, size_t idx) {
  if (S) {
    prefetch_l2(in.hi + idx);
    prefetch_l2(in.lo + idx);
  }
  if (Wp) prefetch_l2(in.w + idx);
  prefetch_l2(in.diag + idx);
  if (in.pf0) prefetch_l2(in.pf0 + idx);
  if (in.pf1) prefetch_l2(in.pf1 + idx);
}

// Parts of the operand at one index.
template <bool S, bool Wp>
struct Parts {
  float2 h, l, w;
};

template <bool S, bool Wp>
__device__ __forceinline__ Parts<S, Wp> load_parts(const MixedIn &in, size_t idx, bool ok) {
  Parts<S, Wp> p;
  const float2 z = make_float2(0.f, 0.f);
  p.h = z;
  p.l = z;
  p.w = z;
  if (ok) {
    if (S) {
      p.h = __ldg(in.hi + idx);
      p.l = __ldg(in.lo + idx);
    }
    if (Wp) p.w = __ldg(in.w + idx);
  }
  return p;
}

template <bool S, bool Wp>
__device__ __forceinline__ float2 value(const Parts<S, Wp> &p, float ws) {
  float2 v = make_float2(0.f, 0.f);
  if (S) {
    v.x = p.l.x;
    v.y = p.l.y;
  }
  if (Wp) {
    v.x = fmaf(ws, p.w.x, v.x);
    v.y = fmaf(ws, p.w.y, v.y);
  }
  if (S) {
    v.x += p.h.x;
    v.y += p.h.y;
  }
  return v;
}

// a - c, part by part.
template <bool S, bool Wp>
__device__ __forceinline__ float2 diff(const Parts<S, Wp> &a, const Parts<S, Wp> &c, float ws) {
  float2 d = make_float2(0.f, 0.f);
  if (Wp) {
    d.x = ws * (a.w.x - c.w.x);
    d.y = ws * (a.w.y - c.w.y);
  }
  if (S) {
    d.x += (a.l.x - c.l.x);
    d.y += (a.l.y - c.l.y);
    d.x += (a.h.x - c.h.x);
    d.y += (a.h.y - c.h.y);
  }
  return d;
}

// Split an FP64 value into hi + lo (two FP32 parts).
__device__ __forceinline__ void split2(double2 v, float2 &h, float2 &lo) {
  h = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
  lo = make_float2(__double2float_rn(v.x - (double)h.x), __double2float_rn(v.y - (double)h.y));
}

// Walk rows [l0, l1) of column i and call f(i, idx, Hx, x_center).  PF > 0
// asks L2 for the operand and diagonal rows PF rows ahead.
// VG: velocity gauge, (A/c) p_z with p_z = -i [ (d/dr - l/r) kappa_l f_{l-1}
// + (d/dr + (l+1)/r) kappa_{l+1} f_{l+1} ] (the partial-wave form of -i d/dz;
// the paper prints the l/r terms with the opposite signs) in place of r E kappa.
// CG: the operand's loads go to L2 (see ldx).
template <int ST, int PF = 0, bool SCALED = false, bool VG = false, bool CG = false, typename F>
__device__ __forceinline__ void walk_rows(const StencilIn &in, int i, int l0, int l1, F &&f) {
  static_assert(!(VG && CG), "the velocity gauge's first derivatives read through the read-only path");
  const int N = in.N, L = in.L;
  const double2 z = make_double2(0.0, 0.0);
  const double Er = __dmul_rn(in.E, in.rj[i]);
  double2 prev = (l0 > 0) ? ldx<CG>(in.x + (size_t)(l0 - 1) * N + i) : z;
  double2 cur = ldx<CG>(in.x + (size_t)l0 * N + i);
  double a_cur = __dmul_rn(in.kappa[l0], Er);
  if (PF > 0)
    for (int q = 1; q < PF && l0 + q < l1; ++q) {
      prefetch_l2(in.x + (size_t)(l0 + q) * N + i);
      prefetch_l2(in.diag + (size_t)(l0 + q) * N + i);
    }
  for (int l = l0; l < l1; ++l) {
    const size_t idx = (size_t)l * N + i;
    if (PF > 0 && l + PF < l1) {
      prefetch_l2(in.x + idx + (size_t)PF * N);
      prefetch_l2(in.diag + idx + (size_t)PF * N);
    }
    const double2 next = (l < L) ? ldx<CG>(in.x + idx + N) : z;
    const double a_next = __dmul_rn(in.kappa[l + 1], Er);
    const double d = SCALED ? __dmul_rn(in.dscale, __ldg(in.diag + idx)) : __ldg(in.diag + idx);
    double2 t = h_point<ST, !VG, CG>(in, in.x + (size_t)l * N, i, d, prev, cur, next, a_cur, a_next);
    if (VG) {
      const double ri = __ldg(in.rinv + i);
      double wx = 0.0, wy = 0.0;
      if (l > 0) {
        const double2 dp = d1_point<ST>(in, in.x + (size_t)(l - 1) * N, i);
        const double k = in.kappa[l], lr = __dmul_rn((double)l, ri);
        wx = __dmul_rn(k, __fma_rn(-lr, prev.x, dp.x));
        wy = __dmul_rn(k, __fma_rn(-lr, prev.y, dp.y));
      }
      if (l < L) {
        const double2 dn = d1_point<ST>(in, in.x + (size_t)(l + 1) * N, i);
        const double k = in.kappa[l + 1], lr = __dmul_rn((double)(l + 1), ri);
        wx = __fma_rn(k, __fma_rn(lr, next.x, dn.x), wx);
        wy = __fma_rn(k, __fma_rn(lr, next.y, dn.y), wy);
      }
      // -i (A/c) w
      t.x = __fma_rn(in.E, wy, t.x);
      t.y = __fma_rn(-in.E, wx, t.y);
    }
    f(i, idx, t, cur);
    prev = cur;
    cur = next;
    a_cur = a_next;
  }
}

// First derivative of the mixed operand's row starting at element `row`, at
// column i (zero beyond the box): the formula of d1_point, with each
// difference formed part by part (diff) as in the Laplacian.
template <int ST, bool S, bool Wp>
__device__ __forceinline__ float2 mixed_d1(const MixedIn &in, size_t row, int i) {
  const Parts<S, Wp> m1 = load_parts<S, Wp>(in, row + i - 1, i >= 1);
  const Parts<S, Wp> p1 = load_parts<S, Wp>(in, row + i + 1, i + 1 < in.N);
  const float2 d1 = diff(p1, m1, in.ws);
  if (ST == 5) {
    const Parts<S, Wp> m2 = load_parts<S, Wp>(in, row + i - 2, i >= 2);
    const Parts<S, Wp> p2 = load_parts<S, Wp>(in, row + i + 2, i + 2 < in.N);
    const float2 d2 = diff(m2, p2, in.ws);
    return make_float2(in.d1c * fmaf(8.f, d1.x, d2.x), in.d1c * fmaf(8.f, d1.y, d2.y));
  }
  return make_float2(in.d1c * d1.x, in.d1c * d1.y);
}

// Walk rows [l0, l1) of column i of the mixed operand; f(i, idx, Hx, x_center).
// PF > 0 asks L2 for every operand row PF rows ahead (prefetch_row).
// VG: the velocity-gauge coupling (A/c) p_z of walk_rows in place of r E kappa.
template <int ST, bool S, bool Wp, int PF = kPrefetchRows, bool VG = false, typename F>
__device__ __forceinline__ void mixed_walk_rows(const MixedIn &in, int i, int l0, int l1, F &&f) {
  const int N = in.N, L = in.L;
  const float Er = in.E * in.rj[i];
  Parts<S, Wp> prev = load_parts<S, Wp>(in, (size_t)(l0 - 1) * N + i, l0 > 0);
  Parts<S, Wp> cur = load_parts<S, Wp>(in, (size_t)l0 * N + i, true);
  float a_cur = in.kappa[l0] * Er;
  if (PF > 0)
    for (int q = 1; q < PF && l0 + q < l1; ++q) prefetch_row<S, Wp>(in, (size_t)(l0 + q) * N + i);
  for (int l = l0; l < l1; ++l) {
    const size_t idx = (size_t)l * N + i;
    if (PF > 0 && l + PF < l1) prefetch_row<S, Wp>(in, idx + (size_t)PF * N);
    const Parts<S, Wp> next = load_parts<S, Wp>(in, idx + N, l < L);
    const float a_next = in.kappa[l + 1] * Er;
    const Parts<S, Wp> m1 = load_parts<S, Wp>(in, idx - 1, i >= 1);
    const Parts<S, Wp> p1 = load_parts<S, Wp>(in, idx + 1, i + 1 < N);
    const float2 d1m = diff(m1, cur, in.ws), d1p = diff(p1, cur, in.ws);
    const float2 vc = value(cur, in.ws), vp = value(prev, in.ws), vn = value(next, in.ws);
    const float dg = __ldg(in.diag + idx);
    float tx = in.c1 * (d1m.x + d1p.x);
    float ty = in.c1 * (d1m.y + d1p.y);
    if (ST == 5) {
      const Parts<S, Wp> m2 = load_parts<S, Wp>(in, idx - 2, i >= 2);
      const Parts<S, Wp> p2 = load_parts<S, Wp>(in, idx + 2, i + 2 < N);
      const float2 d2m = diff(m2, cur, in.ws), d2p = diff(p2, cur, in.ws);
      tx = fmaf(in.c2, d2m.x + d2p.x, tx);
      ty = fmaf(in.c2, d2m.y + d2p.y, ty);
    }
    tx = fmaf(dg, vc.x, tx);
    ty = fmaf(dg, vc.y, ty);
    if (VG) {
      const float ri = in.rinv[i];
      float wx = 0.f, wy = 0.f;
      if (l > 0) {
        const float2 dp = mixed_d1<ST, S, Wp>(in, (size_t)(l - 1) * N, i);
        const float k = in.kappa[l], lr = (float)l * ri;
        wx = k * fmaf(-lr, vp.x, dp.x);
        wy = k * fmaf(-lr, vp.y, dp.y);
      }
      if (l < L) {
        const float2 dn = mixed_d1<ST, S, Wp>(in, (size_t)(l + 1) * N, i);
        const float k = in.kappa[l + 1], lr = (float)(l + 1) * ri;
        wx = fmaf(k, fmaf(lr, vn.x, dn.x), wx);
        wy = fmaf(k, fmaf(lr, vn.y, dn.y), wy);
      }
      // -i (A/c) w
      tx = fmaf(in.E, wy, tx);
      ty = fmaf(-in.E, wx, ty);
    } else {
      tx = fmaf(a_cur, vp.x, tx);
      ty = fmaf(a_cur, vp.y, ty);
      tx = fmaf(a_next, vn.x, tx);
      ty = fmaf(a_next, vn.y, ty);
    }
    f(i, idx, make_float2(tx, ty), vc);
    prev = cur;
    cur = next;
    a_cur = a_next;
  }
}


}  // namespace stencil
}  // namespace tdse_dev
