// Point evaluators of the Hamiltonian shared by the single-instance and the
// batched kernels: the FP64 stencil (Sec. 2, Eq. (h_matrix) of arXiv 1308.1856)
// and the mixed-precision operand (FP32 parts, difference-form Laplacian).
#pragma once

#include <cuda_runtime.h>

namespace tdse_dev {
namespace stencil {

__device__ __forceinline__ double2 ldg2(const double2 *p) { return __ldg(p); }

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
template <int ST, bool LG = true>
__device__ __forceinline__ double2 h_point(const StencilIn &in, const double2 *row, int i,
                                           double d, double2 prev, double2 cur, double2 next,
                                           double a_cur, double a_next) {
  const double2 z = make_double2(0.0, 0.0);
  const double2 m1 = (i >= 1) ? ldg2(row + i - 1) : z;
  const double2 p1 = (i + 1 < in.N) ? ldg2(row + i + 1) : z;
  double tx = __dmul_rn(d, cur.x);
  double ty = __dmul_rn(d, cur.y);
  tx = __fma_rn(in.c1, __dadd_rn(m1.x, p1.x), tx);
  ty = __fma_rn(in.c1, __dadd_rn(m1.y, p1.y), ty);
  if (ST == 5) {
    const double2 m2 = (i >= 2) ? ldg2(row + i - 2) : z;
    const double2 p2 = (i + 2 < in.N) ? ldg2(row + i + 2) : z;
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
template <int ST, int PF = 0, bool SCALED = false, bool VG = false, typename F>
__device__ __forceinline__ void walk_rows(const StencilIn &in, int i, int l0, int l1, F &&f) {
  const int N = in.N, L = in.L;
  const double2 z = make_double2(0.0, 0.0);
  const double Er = __dmul_rn(in.E, in.rj[i]);
  double2 prev = (l0 > 0) ? ldg2(in.x + (size_t)(l0 - 1) * N + i) : z;
  double2 cur = ldg2(in.x + (size_t)l0 * N + i);
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
    const double2 next = (l < L) ? ldg2(in.x + idx + N) : z;
    const double a_next = __dmul_rn(in.kappa[l + 1], Er);
    const double d = SCALED ? __dmul_rn(in.dscale, __ldg(in.diag + idx)) : __ldg(in.diag + idx);
    double2 t = h_point<ST, !VG>(in, in.x + (size_t)l * N, i, d, prev, cur, next, a_cur, a_next);
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


// ---------------------------------------------------------------------------
// Staged walk of the mixed operand: the same arithmetic as mixed_walk_rows,
// with the rows brought into a per-warp ring of shared memory by cp.async
// (LDGSTS) D rows ahead, so that D rows of loads are in flight per warp
// without holding registers.  A ring slot holds one row of the warp's
// 32-column group: each operand part with a two-column halo on both sides
// (36 complex64 values), the 32 diagonal values and NE extra complex64 rows
// that the caller's epilogue reads at the same index (f gets them as e0, e1).
// Rows outside [0, L] and columns outside [0, N) read as zero.
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// 8- or 4-byte asynchronous copy global -> shared; ok = false writes zeros
// (source size 0: nothing is read, src is only a valid placeholder).
__device__ __forceinline__ void cp_async8(void *dst, const void *src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(ok ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(ok ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <bool S, bool Wp, int NE>
struct RingLayout {
  static constexpr int kH = 0;                        // float2 offsets inside a slot
  static constexpr int kL = kH + (S ? 36 : 0);
  static constexpr int kW = kL + (S ? 36 : 0);
  static constexpr int kE = kW + (Wp ? 36 : 0);
  static constexpr int kD = kE + 32 * NE;             // 32 floats = 16 float2
  static constexpr int kSlot = kD + 16;               // float2 per slot
};

// Shared memory (bytes) of one warp's ring of depth D.
template <bool S, bool Wp, int NE, int D>
constexpr int ring_bytes() { return (D + 1) * RingLayout<S, Wp, NE>::kSlot * 8; }

template <bool S, bool Wp>
__device__ __forceinline__ Parts<S, Wp> ring_parts(const float2 *slot, int c) {
  using RL = RingLayout<S, Wp, 0>;
  Parts<S, Wp> p;
  const float2 z = make_float2(0.f, 0.f);
  p.h = S ? slot[RL::kH + c] : z;
  p.l = S ? slot[RL::kL + c] : z;
  p.w = Wp ? slot[RL::kW + c] : z;
  return p;
}

// Walk rows [l0, l1) of column group jg; every lane of the warp must call it
// (lanes whose column is >= N only help with the copies).  ring points at the
// warp's D + 1 slots.  f(i, idx, Hx, x_center, e0, e1).
template <int ST, bool S, bool Wp, int NE, int D, typename F>
__device__ __forceinline__ void staged_walk_rows(const MixedIn &in, float2 *ring, int jg, int l0, int l1, F &&f) {
  static_assert(D >= 2, "ring depth");
  using RL = RingLayout<S, Wp, NE>;
  constexpr int R = D + 1;
  const int lane = threadIdx.x & 31;
  const int N = in.N, L = in.L;
  const int j0 = jg * 32;
  const int i = j0 + lane;
  const bool active = i < N;
  const int last = min(l1, L);   // the last row read (the next row of l1 - 1)
  // halo columns: lanes 0, 1 -> j0 - 2, j0 - 1 (entries 0, 1); lanes 2, 3 -> j0 + 32, j0 + 33 (34, 35)
  const int hc = (lane < 2) ? j0 - 2 + lane : j0 + 30 + lane;
  const int he = (lane < 2) ? lane : 32 + lane;
  const bool hok = lane < 4 && hc >= 0 && hc < N;
  auto slot_of = [&](int row) { return ring + ((row % R + R) % R) * RL::kSlot; };
  auto issue = [&](int row) {
    float2 *sl = slot_of(row);
    if (row >= 0 && row <= last) {
      const size_t base = (size_t)row * N;
      const size_t ci = base + (active ? i : 0);
      const size_t ch = base + (hok ? hc : 0);
      if (S) {
        cp_async8(sl + RL::kH + 2 + lane, in.hi + ci, active);
        cp_async8(sl + RL::kL + 2 + lane, in.lo + ci, active);
        if (lane < 4) {
          cp_async8(sl + RL::kH + he, in.hi + ch, hok);
          cp_async8(sl + RL::kL + he, in.lo + ch, hok);
        }
      }
      if (Wp) {
        cp_async8(sl + RL::kW + 2 + lane, in.w + ci, active);
        if (lane < 4) cp_async8(sl + RL::kW + he, in.w + ch, hok);
      }
      if (row < l1) {   // the diagonal and the epilogue rows only for computed rows
        cp_async4(reinterpret_cast<float *>(sl + RL::kD) + lane, in.diag + ci, active);
        if (NE > 0) cp_async8(sl + RL::kE + lane, in.pf0 + ci, active);
        if (NE > 1) cp_async8(sl + RL::kE + 32 + lane, in.pf1 + ci, active);
      }
    } else if (row >= l0 - 1 && row <= l1) {
      // a row outside [0, L] read as prev or next: zero operand parts
      const float2 z = make_float2(0.f, 0.f);
      if (S) {
        sl[RL::kH + 2 + lane] = z;
        sl[RL::kL + 2 + lane] = z;
        if (lane < 4) {
          sl[RL::kH + he] = z;
          sl[RL::kL + he] = z;
        }
      }
      if (Wp) {
        sl[RL::kW + 2 + lane] = z;
        if (lane < 4) sl[RL::kW + he] = z;
      }
    }
    cp_async_commit();
  };
  const float Er = active ? in.E * in.rj[i] : 0.f;
  for (int q = -1; q < D; ++q) issue(l0 + q);
  float a_cur = in.kappa[l0] * Er;
  for (int l = l0; l < l1; ++l) {
    cp_async_wait<D - 2>();   // rows up to l + 1 have landed
    __syncwarp();
    const float a_next = in.kappa[l + 1] * Er;
    if (active) {
      const float2 *sp = slot_of(l - 1), *sc = slot_of(l), *sn = slot_of(l + 1);
      const Parts<S, Wp> prev = ring_parts<S, Wp>(sp + 0, 2 + lane);
      const Parts<S, Wp> cur = ring_parts<S, Wp>(sc, 2 + lane);
      const Parts<S, Wp> next = ring_parts<S, Wp>(sn, 2 + lane);
      const Parts<S, Wp> m1 = ring_parts<S, Wp>(sc, 1 + lane);
      const Parts<S, Wp> p1 = ring_parts<S, Wp>(sc, 3 + lane);
      const float2 d1m = diff(m1, cur, in.ws), d1p = diff(p1, cur, in.ws);
      const float2 vc = value(cur, in.ws), vp = value(prev, in.ws), vn = value(next, in.ws);
      const float dg = reinterpret_cast<const float *>(sc + RL::kD)[lane];
      float tx = in.c1 * (d1m.x + d1p.x);
      float ty = in.c1 * (d1m.y + d1p.y);
      if (ST == 5) {
        const Parts<S, Wp> m2 = ring_parts<S, Wp>(sc, lane);
        const Parts<S, Wp> p2 = ring_parts<S, Wp>(sc, 4 + lane);
        const float2 d2m = diff(m2, cur, in.ws), d2p = diff(p2, cur, in.ws);
        tx = fmaf(in.c2, d2m.x + d2p.x, tx);
        ty = fmaf(in.c2, d2m.y + d2p.y, ty);
      }
      tx = fmaf(dg, vc.x, tx);
      ty = fmaf(dg, vc.y, ty);
      tx = fmaf(a_cur, vp.x, tx);
      ty = fmaf(a_cur, vp.y, ty);
      tx = fmaf(a_next, vn.x, tx);
      ty = fmaf(a_next, vn.y, ty);
      const float2 z = make_float2(0.f, 0.f);
      const float2 e0 = NE > 0 ? sc[RL::kE + lane] : z;
      const float2 e1 = NE > 1 ? sc[RL::kE + 32 + lane] : z;
      f(i, (size_t)l * N + i, make_float2(tx, ty), vc, e0, e1);
    }
    a_cur = a_next;
    __syncwarp();             // every lane is done with row l - 1's slot
    issue(l + D);             // reuses it
  }
  cp_async_wait<0>();
  __syncwarp();
}

}  // namespace stencil
}  // namespace tdse_dev
