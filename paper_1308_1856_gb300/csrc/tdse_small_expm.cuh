// exp(-i T dt) e_1 for the Lanczos tridiagonal T (one block, k <= 32).
//
// The Lanczos propagator (arXiv 1308.1856, Sec. 5 "Lanczos.c" and Appendix
// "Lanczos methods") needs c = exp(-i T dt) e_1 for the real symmetric
// tridiagonal T = tridiag(beta, alpha, beta) of the current step; the paper
// forms it with a short Taylor series in one work group ("Taylor1").  That
// series is unusable when ||T|| dt is large (the stiff grids of this library
// reach ||T|| dt ~ 1e4), so c is formed from the eigendecomposition
// T = X diag(lambda) X^T:  c_i = sum_e X_ie X_0e exp(-i lambda_e dt).
//
// On GB300 a dependent FP64 instruction costs ~64 cycles (FP64 divide and
// square root ~650), so a serial FP64 eigen-solver would take hundreds of
// microseconds.  Instead:
//   1. an FP32 cyclic Jacobi method (k/2 rotations per round in parallel,
//      round-robin pairing, one warp) gives an orthonormal basis accurate to
//      FP32 rounding (eigenvectors of close eigenvalues only to ~1e-3);
//   2. Ogita-Aishima refinement iterations in FP64 (at least two, more
//      until the correction is negligible; matrix products,
//      i.e. parallel DFMA throughput rather than latency) make X orthonormal
//      and the eigenvalues accurate to FP64 rounding; pairs closer than the
//      iteration's cluster bound are only orthogonalised;
//   3. phases exp(-i lambda dt) in FP64, with a first-order correction for
//      what the refinement leaves off the diagonal of X^T T X (rounding and
//      the coupling inside eigenvalue clusters it cannot separate); one
//      sincos per eigenvalue, the divided differences from those (or a
//      short series where they would cancel).
// Barriers, not arithmetic, set the time of a block this small: the Jacobi
// rounds run in one warp (__syncwarp only) and a refinement iteration has
// four block barriers.
// The breakdown rule beta_j <= 1e-13 max(1, max_{i<=j} |alpha_i|) fixes k.
//
// This header holds the one-block body (expm_body, 256 threads); it is
// included by the single-block launchers and by the cluster kernel of small
// grids, which runs it inside its own launch.
#pragma once

#include <cuda_runtime.h>

#include "tdse_internal.cuh"

namespace tdse_dev {

namespace {

constexpr int kEx = 256;
constexpr int KP = kMaxKrylov;
constexpr int kRefineIters = 2;      // refinement iterations always run
constexpr int kRefineMax = 12;       // and at most this many, while the correction is not negligible
// An iteration whose correction E has ||E||_F <= kRefineDone leaves X
// orthonormal and the eigenvalues converged to FP64 rounding (the next
// correction would be O(||E||^2)).  From an FP32 start (error ~1e-7) the
// first correction is ~1e-7 and the second ~1e-14, after which X is exact to
// rounding.  When the FP32 start mixes eigenvectors whose eigenvalues lie
// within FP32 rounding of ||T|| of each other (stiff T: ||T|| ~ 1e5 and
// eigenvalues ~ 1 apart), the first corrections are O(1) and two iterations
// do not converge; the extra ones do.
constexpr float kRefineDone = 1e-9f;

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace

// Thread mappings below use a row stride of 32 (w >> 5, w & 31) so that no
// loop needs a runtime integer division; a row's 32 entries then lie in one
// warp (its lanes), so row sums are warp shuffles.
// imag: c = exp(-T dt) e_1 (imaginary time) instead of exp(-i T dt) e_1.
// The block barrier of the body: the whole CTA of kEx threads, or (named
// barrier 1) the first kEx threads of a larger block that runs the body in
// those threads alone.
struct ExBlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct ExNamedSync {
  __device__ __forceinline__ void operator()() const { asm volatile("bar.sync 1, %0;" ::"n"(kEx) : "memory"); }
};

template <typename Sync = ExBlockSync>
__device__ __forceinline__ void expm_body(int m, double dt, LanczosScalars *ls, bool imag = false,
                                          Sync sync = Sync()) {
  __shared__ double al[KP], be[KP];
  __shared__ float ad[KP], bd[KP];      // FP32 diagonal and couplings of T during the QR steps
  __shared__ float Vf[KP][KP + 1];
  __shared__ double X0[KP][KP + 1], X1[KP][KP + 1], W[KP][KP + 1], R[KP][KP + 1];
  __shared__ double lam[KP];
  __shared__ double2 hph[KP];          // exp(-i d_a dt / 2) (imaginary time: exp(-d_a dt / 2), 0)
  __shared__ float wpart[kEx / 32][2], wpart2[kEx / 32];
  __shared__ double vr[KP], vi[KP];
  __shared__ unsigned short tri[KP * (KP + 1) / 2];
  __shared__ int s_k;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // ---- Krylov dimension (breakdown rule, decided in FP64) -----------------
  if (tid < 32) {
    const double a = (tid < m) ? ls->alpha[tid] : 0.0;
    const double b = (tid < m - 1) ? ls->beta[tid] : 0.0;
    al[tid] = a;
    be[tid] = b;
    double amax = fabs(a);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double v = __shfl_up_sync(0xffffffffu, amax, o);
      if (tid >= o) amax = fmax(amax, v);
    }
    const bool brk = (tid < m - 1) && (b <= 1e-13 * fmax(1.0, amax));
    const unsigned bm = __ballot_sync(0xffffffffu, brk);
    if (tid == 0) s_k = bm ? __ffs(bm) : m;
  }
  sync();
  const int k = s_k;

  // ---- FP32 eigendecomposition: implicit symmetric QR, in warp 0 ---------
  // Shifted QR steps (Wilkinson shift from the trailing 2x2 of the active
  // block) chase the bulge down the tridiagonal with plane rotations
  // R = [c s; -s c] on rows and columns (i, i+1), T <- R T R^T, and the basis
  // follows, V <- V R^T.  Every lane carries the same scalar chase in
  // registers, and lane r row r of V.  A coupling
  // b_{i-1} with |b_{i-1}| <= eps (|a_{i-1}| + |a_i|) splits the matrix; the
  // lanes test all couplings at once (a ballot), so the active block costs
  // no scan.  The result is accurate to FP32 rounding, as the refinement
  // below needs.
  for (int w = tid; w < KP * 32; w += kEx) {
    const int i = w >> 5, j = w & 31;
    Vf[i][j] = (i == j) ? 1.f : 0.f;
  }
  if (tid < KP) {
    ad[tid] = (tid < k) ? (float)al[tid] : 0.f;
    bd[tid] = (tid + 1 < k) ? (float)be[tid] : 0.f;
  }
  sync();
  if (warp == 0 && k > 1) {
    constexpr float eps = 1.2e-7f;
    int m = k - 1;
    for (int step = 0; step < 30 * k; ++step) {
      bool small = false;
      if (lane >= 1 && lane < k) small = fabsf(bd[lane - 1]) <= eps * (fabsf(ad[lane - 1]) + fabsf(ad[lane]));
      const unsigned neg = __ballot_sync(0xffffffffu, small);
      const unsigned upto = (m >= 31) ? 0xffffffffu : ((2u << m) - 1u);
      const unsigned live = ~neg & upto & ~1u;   // bit i: the coupling of i-1 and i, i <= m, is still there
      if (!live) break;
      m = 31 - __clz(live);                      // bottom of the lowest unreduced block
      const unsigned below = neg & ((1u << m) - 1u) & ~1u;
      const int l = below ? 31 - __clz(below) : 0;   // its top
      // Wilkinson shift (any shift keeps the step exact; this one converges fast)
      const float am1 = ad[m - 1], am = ad[m], bm = bd[m - 1];
      const float dd = 0.5f * (am1 - am);
      const float den = dd + copysignf(sqrtf(fmaf(dd, dd, bm * bm)), dd);
      const float mu = am - __fdividef(bm * bm, den);
      // the chase over [l, m], in registers: the next rotation's entries of T
      // and of lane r's row of V are loaded one rotation ahead, so no load
      // waits inside the chain; every lane stores the same values of T
      float ak = ad[l], ak1 = ad[l + 1], bk = bd[l];
      float bk1n = (l + 1 < m) ? bd[l + 1] : 0.f, ak2n = (l + 2 <= m) ? ad[l + 2] : 0.f;
      const int vr_ = (lane < k) ? lane : 0;                // rows past k: a harmless copy of row 0
      float v0 = Vf[vr_][l], w1n = Vf[vr_][l + 1];
      float x = ak - mu, z = bk;
      for (int i = l; i < m; ++i) {
        const float bk1 = bk1n, ak2 = ak2n, w1 = w1n;    // b_{i+1} (0 past the block), a_{i+2}, V[r][i+1]
        bk1n = (i + 2 < m) ? bd[i + 2] : 0.f;
        ak2n = (i + 3 <= m) ? ad[i + 3] : 0.f;
        w1n = (i + 2 <= m) ? Vf[vr_][i + 2] : 0.f;
        const float h2 = fmaf(x, x, z * z);
        const float rr = rsqrtf(h2);
        const bool nz = h2 > 0.f;
        const float c = nz ? x * rr : 1.f, sn = nz ? z * rr : 0.f, r = nz ? h2 * rr : 0.f;
        const float c2 = c * c, s2 = sn * sn, cs = c * sn;
        const float na = fmaf(c2, ak, fmaf(2.f * cs, bk, s2 * ak1));
        const float na1 = fmaf(s2, ak, fmaf(-2.f * cs, bk, c2 * ak1));
        const float nb = fmaf(cs, ak1 - ak, (c2 - s2) * bk);
        ad[i] = na;
        if (i > l) bd[i - 1] = r;                          // the bulge is gone: b_{i-1} = r
        if (lane < k) Vf[lane][i] = fmaf(c, v0, sn * w1);
        v0 = fmaf(-sn, v0, c * w1);
        // the next rotation zeroes the new bulge s b_{i+1} against t_{i+1,i}
        x = nb;
        z = sn * bk1;
        ak = na1;
        bk = c * bk1;
        ak1 = ak2;
      }
      ad[m] = ak;
      bd[m - 1] = x;
      if (lane < k) Vf[lane][m] = v0;
      __syncwarp();
    }
  }
  sync();

  // ---- FP64 Ogita-Aishima refinement -------------------------------------
  // An FP64 warp instruction holds its SM sub-partition's FP64 pipe for the
  // same time whatever number of lanes it has active, so every FP64 pass
  // below packs its items densely into consecutive threads (item w of the
  // k x k set is (w / k, w mod k)), and the dot products of R and S are split
  // over P lanes where the items alone would leave lanes idle.  X alternates
  // between two buffers (the update reads the old one); during an iteration
  // the new buffer first holds S = X^T T X.
  double (*Xc)[KP + 1] = X0;
  double (*Xn)[KP + 1] = X1;
  const int kk = k * k;
  const unsigned kinv = (65536u + (unsigned)k - 1u) / (unsigned)k;   // w / k = (w kinv) >> 16 for w < 1024
  const int nt = k * (k + 1) / 2;                                    // upper-triangle items a <= b
  const int lp = (4 * nt <= kEx) ? 2 : ((2 * nt <= kEx) ? 1 : 0);    // P = 2^lp lanes per R, S item
  const int P = 1 << lp;
  if (tid < k) {
    const int base = tid * k - tid * (tid - 1) / 2;
    for (int b = tid; b < k; ++b) tri[base + b - tid] = (unsigned short)(tid | (b << 8));
  }
  for (int w = tid; w < kk; w += kEx) {
    const int i = (int)(((unsigned)w * kinv) >> 16), j = w - i * k;
    Xc[i][j] = (double)Vf[i][j];
  }
  // ||T||_F in FP32 (the scale of a threshold), the same fixed-order sum in every thread
  float tn2 = 0.f;
  for (int i = 0; i < k; ++i) {
    tn2 = fmaf((float)al[i], (float)al[i], tn2);
    if (i + 1 < k) tn2 = fmaf(2.f * (float)be[i], (float)be[i], tn2);
  }
  const double tnorm = (double)sqrtf(tn2);
  sync();
  for (int it = 0; it < kRefineMax; ++it) {
    // W = T X
    for (int w = tid; w < kk; w += kEx) {
      const int i = (int)(((unsigned)w * kinv) >> 16), e = w - i * k;
      double v = al[i] * Xc[i][e];
      if (i > 0) v = fma(be[i - 1], Xc[i - 1][e], v);
      if (i + 1 < k) v = fma(be[i], Xc[i + 1][e], v);
      W[i][e] = v;
    }
    sync();
    // R = I - X^T X and S = X^T T X are symmetric: item (a <= b), its dot
    // products over i = part, part + P, ..., the P parts added by shuffles.
    // lambda_a = S_aa / (1 - R_aa) with |R_aa| <~ 1e-6: 1/(1-r) = 1 + r + r^2 (+ O(1e-18)).
    // The same pass gathers the squares of the cluster bound's norms.
    float sd2 = 0.f, r2 = 0.f;
    for (int g0 = 0; g0 < nt * P; g0 += kEx) {
      const int g = g0 + tid, item = g >> lp, part = g & (P - 1);
      const bool ok = item < nt;
      int a = 0, b = 0;
      if (ok) {
        const unsigned ab = tri[item];
        a = (int)(ab & 0xffu);
        b = (int)(ab >> 8);
      }
      double r0 = 0.0, r1 = 0.0, s0 = 0.0, s1 = 0.0;
      if (ok) {
        int i = part;
        for (; i + P < k; i += 2 * P) {
          r0 = fma(Xc[i][a], Xc[i][b], r0);
          s0 = fma(Xc[i][a], W[i][b], s0);
          r1 = fma(Xc[i + P][a], Xc[i + P][b], r1);
          s1 = fma(Xc[i + P][a], W[i + P][b], s1);
        }
        if (i < k) {
          r0 = fma(Xc[i][a], Xc[i][b], r0);
          s0 = fma(Xc[i][a], W[i][b], s0);
        }
      }
      double rs = r0 + r1, ss = s0 + s1;
      for (int o = 1; o < P; o <<= 1) {
        rs += __shfl_xor_sync(0xffffffffu, rs, o);
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
      }
      if (ok && part == 0) {
        const double rr = ((a == b) ? 1.0 : 0.0) - rs;
        R[a][b] = rr;
        R[b][a] = rr;
        Xn[a][b] = ss;
        Xn[b][a] = ss;
        const float rf = (float)rr;
        if (a == b) {
          lam[a] = ss * fma(rr, rr, 1.0 + rr);
          const float d = (float)(-ss * fma(rr, rr, rr));   // S_aa - lambda_a
          sd2 = fmaf(d, d, sd2);
          r2 = fmaf(rf, rf, r2);
        } else {
          const float d = (float)ss;
          sd2 = fmaf(2.f * d, d, sd2);
          r2 = fmaf(2.f * rf, rf, r2);
        }
      }
    }
    sd2 = warp_sum_f(sd2);
    r2 = warp_sum_f(r2);
    if (lane == 0) {
      wpart[warp][0] = sd2;
      wpart[warp][1] = r2;
    }
    sync();
    // cluster bound delta = 2 (||S - diag(lambda)|| + ||T|| ||R||) (Frobenius
    // norms): pairs closer than delta are only orthogonalised
    float sdt = 0.f, rt = 0.f;
#pragma unroll
    for (int q = 0; q < kEx / 32; ++q) {
      sdt += wpart[q][0];
      rt += wpart[q][1];
    }
    const double delta = 2.0 * ((double)sqrtf(sdt) + tnorm * (double)sqrtf(rt));
    // E (stored in W); the reciprocal of each gap avoids the ~640-cycle FP64 divide
    float e2 = 0.f;
    for (int w = tid; w < kk; w += kEx) {
      const int a = (int)(((unsigned)w * kinv) >> 16), b = w - a * k;
      double e;
      const double gap = lam[b] - lam[a];
      if (a == b || fabs(gap) <= delta) {
        e = 0.5 * R[a][b];
      } else {
        // FP32 reciprocal of the rounded gap (relative error ~1e-7), then two Newton steps
        double y = (double)__frcp_rn((float)gap);
        y = y * fma(-gap, y, 2.0);
        y = y * fma(-gap, y, 2.0);
        e = fma(lam[b], R[a][b], Xn[a][b]) * y;
      }
      W[a][b] = e;
      e2 = fmaf((float)e, (float)e, e2);
    }
    e2 = warp_sum_f(e2);
    if (lane == 0) wpart2[warp] = e2;
    sync();
    float et = 0.f;
#pragma unroll
    for (int q = 0; q < kEx / 32; ++q) et += wpart2[q];
    const float en = sqrtf(et);
    // X <- X + X E, into the other buffer
    for (int w = tid; w < kk; w += kEx) {
      const int i = (int)(((unsigned)w * kinv) >> 16), b = w - i * k;
      double v0 = Xc[i][b], v1 = 0.0;
      int a = 0;
      for (; a + 1 < k; a += 2) {
        v0 = fma(Xc[i][a], W[a][b], v0);
        v1 = fma(Xc[i][a + 1], W[a + 1][b], v1);
      }
      if (a < k) v0 = fma(Xc[i][a], W[a][b], v0);
      Xn[i][b] = v0 + v1;
    }
    sync();
    double (*xt)[KP + 1] = Xc;
    Xc = Xn;
    Xn = xt;
    if (it + 1 >= kRefineIters && en <= kRefineDone) break;   // uniform: en is the same sum everywhere
  }

  // ---- S = X^T T X of the final basis (orthonormal to FP64 rounding), so that
  // exp(-i T dt) = X exp(-i S dt) X^T.  S = D + F with D its diagonal and F
  // what the refinement leaves off the diagonal: rounding, and the coupling
  // inside eigenvalue clusters closer than its cluster bound, which it never
  // separates (the bound cannot fall below that coupling).  To first order in F
  //   exp(-i S dt) = exp(-i D dt) + Phi o F,  Phi_ab = (f(d_a) - f(d_b)) / (d_a - d_b),
  // the divided differences of f(x) = exp(-i x dt) (exp(-x dt) in imaginary
  // time; the derivative f'(d_a) where d_a = d_b); the O(|F dt|^2) remainder
  // is below rounding.  Only v = (f(D) + Phi o F) y with y_b = X_0b is needed.
  for (int w = tid; w < kk; w += kEx) {
    const int i = (int)(((unsigned)w * kinv) >> 16), e = w - i * k;
    double v = al[i] * Xc[i][e];
    if (i > 0) v = fma(be[i - 1], Xc[i - 1][e], v);
    if (i + 1 < k) v = fma(be[i], Xc[i + 1][e], v);
    W[i][e] = v;
  }
  sync();
  for (int w = tid; w < kk; w += kEx) {      // S into Xn
    const int a = (int)(((unsigned)w * kinv) >> 16), b = w - a * k;
    double s0 = 0.0, s1 = 0.0;
    int i = 0;
    for (; i + 1 < k; i += 2) {
      s0 = fma(Xc[i][a], W[i][b], s0);
      s1 = fma(Xc[i + 1][a], W[i + 1][b], s1);
    }
    if (i < k) s0 = fma(Xc[i][a], W[i][b], s0);
    Xn[a][b] = s0 + s1;
  }
  sync();
  // half-step factors h_a = f(d_a / 2), in one warp (a transcendental costs
  // the same per warp instruction however few lanes it serves; warp 1, as
  // warp 0 sums the rows below)
  if (warp == 1 && lane < k) {
    const double hp = 0.5 * Xn[lane][lane] * dt;
    if (imag) {
      hph[lane] = make_double2(exp(-hp), 0.0);
    } else {
      double sn, cs;
      sincos(hp, &sn, &cs);
      hph[lane] = make_double2(cs, -sn);
    }
  }
  sync();
  // the terms M_ab y_b, into W (re) and R (im)
  for (int w = tid; w < kk; w += kEx) {
    const int a = (int)(((unsigned)w * kinv) >> 16), b = w - a * k;
    const double y = Xc[0][b];
    const double2 ha = hph[a], hb = hph[b];
    double tr, ti;
    if (a == b) {
      // f(d_a) = h_a^2
      tr = fma(ha.x, ha.x, -ha.y * ha.y) * y;
      ti = 2.0 * ha.x * ha.y * y;
    } else {
      const double da = Xn[a][a], db = Xn[b][b], f = Xn[a][b] * y;
      const double x = 0.5 * (da - db) * dt;    // half the phase difference
      const bool near = fabs(x) < 0.5;
      double pr, pi;                             // Phi_ab
      if (!imag) {
        // -i dt h_a h_b sinc(x); sinc by its series sum_n (-x^2)^n / (2n+1)! to
        // n = 8 for |x| < 0.5 (the rest is below rounding), else sin(x) / x with
        // sin(x) = Im(conj(h_a) h_b) (no cancellation for |x| >= 1/2)
        double q;
        if (near) {
          const double z = -x * x;
          q = 1.0 / 355687428096000.0;
          q = fma(q, z, 1.0 / 1307674368000.0);
          q = fma(q, z, 1.0 / 6227020800.0);
          q = fma(q, z, 1.0 / 39916800.0);
          q = fma(q, z, 1.0 / 362880.0);
          q = fma(q, z, 1.0 / 5040.0);
          q = fma(q, z, 1.0 / 120.0);
          q = fma(q, z, 1.0 / 6.0);
          q = fma(q, z, 1.0);
        } else {
          double rx = (double)__frcp_rn((float)x);
          rx = rx * fma(-x, rx, 2.0);
          rx = rx * fma(-x, rx, 2.0);
          q = fma(ha.x, hb.y, -ha.y * hb.x) * rx;
        }
        const double mr = fma(ha.x, hb.x, -ha.y * hb.y), mi = fma(ha.x, hb.y, ha.y * hb.x);   // h_a h_b
        const double g = dt * q;
        pr = g * mi;       // -i g (mr + i mi)
        pi = -g * mr;
      } else if (near) {
        // -dt h_a h_b sinh(x) / x, by the series sum_n x^(2n) / (2n+1)!
        const double z = x * x;
        double q = 1.0 / 355687428096000.0;
        q = fma(q, z, 1.0 / 1307674368000.0);
        q = fma(q, z, 1.0 / 6227020800.0);
        q = fma(q, z, 1.0 / 39916800.0);
        q = fma(q, z, 1.0 / 362880.0);
        q = fma(q, z, 1.0 / 5040.0);
        q = fma(q, z, 1.0 / 120.0);
        q = fma(q, z, 1.0 / 6.0);
        q = fma(q, z, 1.0);
        pr = -dt * ha.x * hb.x * q;
        pi = 0.0;
      } else {
        // (f(d_a) - f(d_b)) / (d_a - d_b) with f(d) = h^2
        const double gap = da - db;
        double rg = (double)__frcp_rn((float)gap);
        rg = rg * fma(-gap, rg, 2.0);
        rg = rg * fma(-gap, rg, 2.0);
        pr = fma(ha.x, ha.x, -hb.x * hb.x) * rg;
        pi = 0.0;
      }
      tr = pr * f;
      ti = pi * f;
    }
    W[a][b] = tr;
    R[a][b] = ti;
  }
  sync();
  // v = row sums (warp 0, lane a), then c = X v
  if (warp == 0) {
    if (lane < k) {
      double v0 = 0.0, v1 = 0.0, u0 = 0.0, u1 = 0.0;
      int b = 0;
      for (; b + 1 < k; b += 2) {
        v0 += W[lane][b];
        u0 += R[lane][b];
        v1 += W[lane][b + 1];
        u1 += R[lane][b + 1];
      }
      if (b < k) {
        v0 += W[lane][b];
        u0 += R[lane][b];
      }
      vr[lane] = v0 + v1;
      vi[lane] = u0 + u1;
    }
    __syncwarp();
    double2 c = make_double2(0.0, 0.0);
    if (lane < k) {
      double cx1 = 0.0, cy1 = 0.0;
      int e = 0;
      for (; e + 1 < k; e += 2) {
        c.x = fma(Xc[lane][e], vr[e], c.x);
        c.y = fma(Xc[lane][e], vi[e], c.y);
        cx1 = fma(Xc[lane][e + 1], vr[e + 1], cx1);
        cy1 = fma(Xc[lane][e + 1], vi[e + 1], cy1);
      }
      if (e < k) {
        c.x = fma(Xc[lane][e], vr[e], c.x);
        c.y = fma(Xc[lane][e], vi[e], c.y);
      }
      c.x += cx1;
      c.y += cy1;
      // psi_new = ||psi|| sum_j c_j q_j = sum_j coef_j U_j with q_j = sigma_j U_j,
      // U_0 = psi and sigma_0 = 1/||psi||.
      if (lane > 0) {
        const double f = ls->psinorm * ls->sigma[lane];
        c.x *= f;
        c.y *= f;
      }
    }
    ls->coef[lane] = c;
    if (lane == 0) ls->kdim = k;
  }
}

}  // namespace tdse_dev
