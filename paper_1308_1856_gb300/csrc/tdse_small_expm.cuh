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
//      round-robin pairing) gives an orthonormal basis accurate to FP32
//      rounding (eigenvectors of close eigenvalues only to ~1e-3);
//   2. Ogita-Aishima refinement iterations in FP64 (at least three, more
//      until the correction is negligible; matrix products,
//      i.e. parallel DFMA throughput rather than latency) make X orthonormal
//      and the eigenvalues accurate to FP64 rounding; pairs closer than the
//      iteration's cluster bound are only orthogonalised;
//   3. phases exp(-i lambda dt) in FP64, with a first-order correction for
//      what the refinement leaves off the diagonal of X^T T X (rounding and
//      the coupling inside eigenvalue clusters it cannot separate).
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
constexpr int kJacobiSweeps = 12;
constexpr int kRefineIters = 3;      // refinement iterations always run
constexpr int kRefineMax = 12;       // and at most this many, while the correction is not negligible
// An iteration whose correction E has ||E||_F <= kRefineDone leaves X
// orthonormal and the eigenvalues converged to FP64 rounding (the next
// correction would be O(||E||^2)).  When the FP32 start mixes eigenvectors
// whose eigenvalues lie within FP32 rounding of ||T|| of each other (stiff T:
// ||T|| ~ 1e5 and eigenvalues ~ 1 apart), the first corrections are O(1) and
// three iterations do not converge; the extra ones do.
constexpr float kRefineDone = 1e-9f;
// FP32 Jacobi stops once the off-diagonal mass is below this fraction of the
// total (off-diagonal norm ~3e-6 relative): the FP64 refinement converges
// quadratically from there (3e-6 -> 1e-11 -> 1e-22, i.e. FP64 rounding; the
// third iteration removes the rounding left by the second).
constexpr float kJacobiTol = 1e-11f;

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP32 block sum (used only for thresholds: 4-cycle adds instead of 64-cycle FP64).
__device__ float block_sum_f(float v, float *sh) {
  const int tid = threadIdx.x;
  v = warp_sum_f(v);
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    float s = (tid < kEx / 32) ? sh[tid] : 0.f;
    s = warp_sum_f(s);
    if (tid == 0) sh[kEx / 32] = s;
  }
  __syncthreads();
  const float r = sh[kEx / 32];
  __syncthreads();
  return r;
}

// Round-robin ("circle") pairing: in round r of an even count n, pair t is
// (0, r+1) for t = 0, else (1 + (r+t) mod (n-1), 1 + (r-t+n-1) mod (n-1)).
__device__ __forceinline__ void pair_of(int r, int t, int n, int &p, int &q) {
  if (t == 0) {
    p = 0;
    q = r % (n - 1) + 1;
  } else {
    p = (r + t) % (n - 1) + 1;
    q = (r - t + (n - 1)) % (n - 1) + 1;
  }
  if (p > q) { const int x = p; p = q; q = x; }
}

}  // namespace

// Thread mappings below use a row stride of 32 (w >> 5, w & 31) so that no
// loop needs a runtime integer division.
// imag: c = exp(-T dt) e_1 (imaginary time) instead of exp(-i T dt) e_1.
__device__ __forceinline__ void expm_body(int m, double dt, LanczosScalars *ls, bool imag = false) {
  __shared__ double al[KP], be[KP];
  __shared__ float Af[KP][KP + 1];
  __shared__ float Vf[KP][KP + 1];
  __shared__ float rc[KP / 2], rs[KP / 2];
  __shared__ int rp[KP / 2], rq[KP / 2];
  __shared__ unsigned char pp_tab[KP - 1][KP / 2], pq_tab[KP - 1][KP / 2];
  __shared__ double X[KP][KP + 1], W[KP][KP + 1], R[KP][KP + 1], S[KP][KP + 1];
  __shared__ double lam[KP];
  __shared__ float shf[kEx / 32 + 1];
  __shared__ int s_k;
  const int tid = threadIdx.x;

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
  __syncthreads();
  const int k = s_k;
  const int n = (k + 1) & ~1;   // even count for the pairing (index k is a dummy if k odd)

  // ---- FP32 Jacobi ------------------------------------------------------
  // round-robin pairing table for every round (no integer division inside the rounds)
  for (int w = tid; w < (n - 1) * (n / 2); w += kEx) {
    const int r = w / (n / 2), t = w - r * (n / 2);
    int p, q;
    pair_of(r, t, n, p, q);
    pp_tab[r][t] = (unsigned char)p;
    pq_tab[r][t] = (unsigned char)q;
  }
  for (int w = tid; w < KP * 32; w += kEx) {
    const int i = w >> 5, j = w & 31;
    float v = 0.f;
    if (i < k && j < k) {
      if (i == j) v = (float)al[i];
      else if (j == i + 1) v = (float)be[i];
      else if (i == j + 1) v = (float)be[j];
    }
    Af[i][j] = v;
    Vf[i][j] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  for (int sweep = 0; sweep < kJacobiSweeps && k > 1; ++sweep) {
    // convergence test on the off-diagonal mass
    float off = 0.f, tot = 0.f;
    for (int w = tid; w < k * 32; w += kEx) {
      const int i = w >> 5, j = w & 31;
      if (j < k) {
        const float v = Af[i][j];
        tot = fmaf(v, v, tot);
        if (i != j) off = fmaf(v, v, off);
      }
    }
    off = block_sum_f(off, shf);
    tot = block_sum_f(tot, shf);
    if (off <= kJacobiTol * tot) break;      // uniform: every thread holds the same sums
    for (int r = 0; r < n - 1; ++r) {
      if (tid < n / 2) {
        const int p = pp_tab[r][tid], q = pq_tab[r][tid];
        float c = 1.f, s = 0.f;
        if (q < k) {
          const float apq = Af[p][q];
          if (apq != 0.f) {
            // rotation that zeroes A[p][q]; the initial guess needs no IEEE rounding
            const float theta = (Af[q][q] - Af[p][p]) * __frcp_rn(2.f * apq);
            const float at = fabsf(theta);
            float t;
            if (at < 1e15f) {
              const float h2 = fmaf(theta, theta, 1.f);
              t = copysignf(__frcp_rn(at + h2 * rsqrtf(h2)), theta);
            } else {
              t = 0.5f * __frcp_rn(theta);
            }
            c = rsqrtf(fmaf(t, t, 1.f));
            s = t * c;
          }
        }
        rp[tid] = p;
        rq[tid] = q;
        rc[tid] = c;
        rs[tid] = s;
      }
      __syncthreads();
      // A <- J^T A  (rows p, q of every pair)
      for (int w = tid; w < (n / 2) * 32; w += kEx) {
        const int t = w >> 5, col = w & 31;
        const int p = rp[t], q = rq[t];
        if (q < k && col < k) {
          const float c = rc[t], s = rs[t];
          const float ap = Af[p][col], aq = Af[q][col];
          Af[p][col] = c * ap - s * aq;
          Af[q][col] = s * ap + c * aq;
        }
      }
      __syncthreads();
      // A <- A J and V <- V J  (columns p, q of every pair)
      for (int w = tid; w < (n / 2) * 32; w += kEx) {
        const int t = w >> 5, row = w & 31;
        const int p = rp[t], q = rq[t];
        if (q < k && row < k) {
          const float c = rc[t], s = rs[t];
          const float ap = Af[row][p], aq = Af[row][q];
          Af[row][p] = c * ap - s * aq;
          Af[row][q] = s * ap + c * aq;
          const float vp = Vf[row][p], vq = Vf[row][q];
          Vf[row][p] = c * vp - s * vq;
          Vf[row][q] = s * vp + c * vq;
        }
      }
      __syncthreads();
    }
  }

  // ---- FP64 Ogita-Aishima refinement -------------------------------------
  for (int w = tid; w < k * 32; w += kEx) {
    const int i = w >> 5, j = w & 31;
    if (j < k) X[i][j] = (double)Vf[i][j];
  }
  float tnorm2 = 0.f;
  for (int i = tid; i < k; i += kEx) {
    tnorm2 += (float)al[i] * (float)al[i];
    if (i + 1 < k) tnorm2 += 2.f * (float)be[i] * (float)be[i];
  }
  const double tnorm = (double)sqrtf(block_sum_f(tnorm2, shf));   // ||T||_F (also syncs X)
  for (int it = 0; it < kRefineMax; ++it) {
    // W = T X
    for (int w = tid; w < k * 32; w += kEx) {
      const int i = w >> 5, e = w & 31;
      if (e < k) {
        double v = al[i] * X[i][e];
        if (i > 0) v = fma(be[i - 1], X[i - 1][e], v);
        if (i + 1 < k) v = fma(be[i], X[i + 1][e], v);
        W[i][e] = v;
      }
    }
    __syncthreads();
    // R = I - X^T X and S = X^T T X are symmetric: compute a <= b, mirror
    for (int w = tid; w < k * 32; w += kEx) {
      const int a = w >> 5, b = w & 31;
      if (b < k && a <= b) {
        double r0 = 0.0, r1 = 0.0, s0 = 0.0, s1 = 0.0;
        int i = 0;
        for (; i + 1 < k; i += 2) {
          r0 = fma(X[i][a], X[i][b], r0);
          s0 = fma(X[i][a], W[i][b], s0);
          r1 = fma(X[i + 1][a], X[i + 1][b], r1);
          s1 = fma(X[i + 1][a], W[i + 1][b], s1);
        }
        if (i < k) {
          r0 = fma(X[i][a], X[i][b], r0);
          s0 = fma(X[i][a], W[i][b], s0);
        }
        const double rr = ((a == b) ? 1.0 : 0.0) - (r0 + r1);
        const double ss = s0 + s1;
        R[a][b] = rr;
        R[b][a] = rr;
        S[a][b] = ss;
        S[b][a] = ss;
      }
    }
    __syncthreads();
    // lambda_a = S_aa / (1 - R_aa) with |R_aa| <~ 1e-6: 1/(1-r) = 1 + r + r^2 (+ O(1e-18))
    if (tid < k) {
      const double r = R[tid][tid];
      lam[tid] = S[tid][tid] * fma(r, r, 1.0 + r);
    }
    __syncthreads();
    // cluster bound delta = 2 (||S - diag(lambda)|| + ||T|| ||R||) (Frobenius norms,
    // FP32 is enough for a threshold): pairs closer than delta are only orthogonalised
    float sd2 = 0.f, r2 = 0.f;
    for (int w = tid; w < k * 32; w += kEx) {
      const int a = w >> 5, b = w & 31;
      if (b < k) {
        const float d = (float)(S[a][b] - ((a == b) ? lam[a] : 0.0));
        const float rr = (float)R[a][b];
        sd2 = fmaf(d, d, sd2);
        r2 = fmaf(rr, rr, r2);
      }
    }
    const float sdn = sqrtf(block_sum_f(sd2, shf));
    const float rn = sqrtf(block_sum_f(r2, shf));
    const double delta = 2.0 * ((double)sdn + tnorm * (double)rn);
    // E (stored in W); the reciprocal of each gap avoids the ~640-cycle FP64 divide
    float e2 = 0.f;
    for (int w = tid; w < k * 32; w += kEx) {
      const int a = w >> 5, b = w & 31;
      if (b < k) {
        double e;
        const double gap = lam[b] - lam[a];
        if (a == b || fabs(gap) <= delta) {
          e = 0.5 * R[a][b];
        } else {
          // FP32 reciprocal of the rounded gap (relative error ~1e-7), then two Newton steps
          double y = (double)__frcp_rn((float)gap);
          y = y * fma(-gap, y, 2.0);
          y = y * fma(-gap, y, 2.0);
          e = fma(lam[b], R[a][b], S[a][b]) * y;
        }
        W[a][b] = e;
        e2 = fmaf((float)e, (float)e, e2);
      }
    }
    const float en = sqrtf(block_sum_f(e2, shf));   // also the barrier before W is read
    // X <- X + X E   (new X into S, then copy)
    for (int w = tid; w < k * 32; w += kEx) {
      const int i = w >> 5, b = w & 31;
      if (b < k) {
        double v0 = X[i][b], v1 = 0.0;
        int a = 0;
        for (; a + 1 < k; a += 2) {
          v0 = fma(X[i][a], W[a][b], v0);
          v1 = fma(X[i][a + 1], W[a + 1][b], v1);
        }
        if (a < k) v0 = fma(X[i][a], W[a][b], v0);
        S[i][b] = v0 + v1;
      }
    }
    __syncthreads();
    for (int w = tid; w < k * 32; w += kEx) {
      const int i = w >> 5, b = w & 31;
      if (b < k) X[i][b] = S[i][b];
    }
    __syncthreads();
    if (it + 1 >= kRefineIters && en <= kRefineDone) break;   // uniform: en is a block sum
  }

  // ---- S = X^T T X of the final basis (orthonormal to FP64 rounding), so that
  // exp(-i T dt) = X exp(-i S dt) X^T.  S = D + F with D its diagonal and F
  // what the refinement leaves off the diagonal: rounding, and the coupling
  // inside eigenvalue clusters closer than its cluster bound, which it never
  // separates (the bound cannot fall below that coupling).  To first order in F
  //   exp(-i S dt) = exp(-i D dt) + Phi o F,  Phi_ab = (f(d_a) - f(d_b)) / (d_a - d_b),
  // the divided differences of f(x) = exp(-i x dt) (exp(-x dt) in imaginary
  // time; the derivative f'(d_a) where d_a = d_b); the O(|F dt|^2) remainder
  // is below rounding.  M = f(D) + Phi o F goes to R (re) and W (im).
  for (int w = tid; w < k * 32; w += kEx) {
    const int i = w >> 5, e = w & 31;
    if (e < k) {
      double v = al[i] * X[i][e];
      if (i > 0) v = fma(be[i - 1], X[i - 1][e], v);
      if (i + 1 < k) v = fma(be[i], X[i + 1][e], v);
      W[i][e] = v;
    }
  }
  __syncthreads();
  for (int w = tid; w < k * 32; w += kEx) {
    const int a = w >> 5, b = w & 31;
    if (b < k) {
      double s0 = 0.0, s1 = 0.0;
      int i = 0;
      for (; i + 1 < k; i += 2) {
        s0 = fma(X[i][a], W[i][b], s0);
        s1 = fma(X[i + 1][a], W[i + 1][b], s1);
      }
      if (i < k) s0 = fma(X[i][a], W[i][b], s0);
      S[a][b] = s0 + s1;
    }
  }
  __syncthreads();
  for (int w = tid; w < k * 32; w += kEx) {
    const int a = w >> 5, b = w & 31;
    if (b < k) {
      const double da = S[a][a], db = S[b][b];
      const double mu = 0.5 * (da + db);
      const double x = 0.5 * (da - db) * dt;      // half the phase difference
      double mr, mi;
      if (imag) {
        double phi;
        if (fabs(x) < 0.5) {
          const double shx = (x == 0.0) ? 1.0 : sinh(x) / x;
          phi = -dt * exp(-mu * dt) * shx;
        } else {
          phi = (exp(-da * dt) - exp(-db * dt)) / (da - db);
        }
        mr = (a == b) ? exp(-da * dt) : phi * S[a][b];
        mi = 0.0;
      } else {
        // -i dt exp(-i mu dt) sinc(x): sinc is bounded, so no cancellation
        const double snc = (x == 0.0) ? 1.0 : sin(x) / x;
        double sn, cs;
        sincos(mu * dt, &sn, &cs);
        if (a == b) {
          mr = cs;
          mi = -sn;
        } else {
          const double f = dt * snc * S[a][b];
          mr = -f * sn;
          mi = -f * cs;
        }
      }
      R[a][b] = mr;
      W[a][b] = mi;
    }
  }
  __syncthreads();
  // v = M y with y_b = X_0b (the first row of X), into rows 0 and 1 of S
  if (tid < k) {
    double vr = 0.0, vi = 0.0;
    for (int b = 0; b < k; ++b) {
      const double y = X[0][b];
      vr = fma(R[tid][b], y, vr);
      vi = fma(W[tid][b], y, vi);
    }
    lam[tid] = vr;
    al[tid] = vi;    // alpha is no longer needed
  }
  __syncthreads();
  if (tid < k) {
    W[0][tid] = lam[tid];
    W[1][tid] = al[tid];
  }
  __syncthreads();
  if (tid < KP) {
    double2 c = make_double2(0.0, 0.0);
    if (tid < k) {
      double cx1 = 0.0, cy1 = 0.0;
      int e = 0;
      for (; e + 1 < k; e += 2) {
        c.x = fma(X[tid][e], W[0][e], c.x);
        c.y = fma(X[tid][e], W[1][e], c.y);
        cx1 = fma(X[tid][e + 1], W[0][e + 1], cx1);
        cy1 = fma(X[tid][e + 1], W[1][e + 1], cy1);
      }
      if (e < k) {
        c.x = fma(X[tid][e], W[0][e], c.x);
        c.y = fma(X[tid][e], W[1][e], c.y);
      }
      c.x += cx1;
      c.y += cy1;
      // psi_new = ||psi|| sum_j c_j q_j = sum_j coef_j U_j with q_j = sigma_j U_j,
      // U_0 = psi and sigma_0 = 1/||psi||.
      if (tid > 0) {
        const double f = ls->psinorm * ls->sigma[tid];
        c.x *= f;
        c.y *= f;
      }
    }
    ls->coef[tid] = c;
    if (tid == 0) ls->kdim = k;
  }
}

}  // namespace tdse_dev
