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
//      round-robin pairing) gives eigenvectors accurate to ~1e-7;
//   2. three Ogita-Aishima refinement iterations in FP64 (matrix products,
//      i.e. parallel DFMA throughput rather than latency) make X orthonormal
//      and the eigenvalues accurate to FP64 rounding; pairs closer than the
//      iteration's cluster bound are only orthogonalised;
//   3. phases exp(-i lambda dt) in FP64.
// The breakdown rule beta_j <= 1e-13 max(1, max_{i<=j} |alpha_i|) fixes k.
#include <cuda_runtime.h>

#include "tdse_internal.cuh"

namespace tdse_dev {

namespace {

constexpr int kEx = 256;
constexpr int KP = kMaxKrylov;
constexpr int kJacobiSweeps = 12;
constexpr int kRefineIters = 3;
// FP32 Jacobi stops once the off-diagonal mass is below this fraction of the
// total (off-diagonal norm ~3e-6 relative): the FP64 refinement converges
// quadratically from there (3e-6 -> 1e-11 -> 1e-22).
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

// a / b for FP64 without the long-latency division: FP32 reciprocal refined by
// two Newton steps (relative error ~1e-16) when b is inside FP32 range.
__device__ __forceinline__ double fast_div(double a, double b) {
  const double ab = fabs(b);
  if (!(ab > 1e-30 && ab < 1e30)) return a / b;
  double y = (double)__frcp_rn((float)b);
  y = y * fma(-b, y, 2.0);
  y = y * fma(-b, y, 2.0);
  return a * y;
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

__global__ void __launch_bounds__(kEx) lanczos_expm_kernel(int m, double dt, LanczosScalars *ls) {
  __shared__ double al[KP], be[KP];
  __shared__ float Af[KP][KP + 1];
  __shared__ float Vf[KP][KP + 1];
  __shared__ float rc[KP / 2], rs[KP / 2];
  __shared__ int rp[KP / 2], rq[KP / 2];
  __shared__ double X[KP][KP + 1], W[KP][KP + 1], R[KP][KP + 1], S[KP][KP + 1];
  __shared__ double lam[KP];
  __shared__ float shf[kEx / 32 + 1];
  __shared__ int s_k, s_done;
  const int tid = threadIdx.x;

  // ---- Krylov dimension (breakdown rule) -------------------------------
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
  for (int w = tid; w < KP * KP; w += kEx) {
    const int i = w / KP, j = w % KP;
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
    for (int w = tid; w < k * k; w += kEx) {
      const int i = w / k, j = w % k;
      const float v = Af[i][j];
      tot += v * v;
      if (i != j) off += v * v;
    }
    off = block_sum_f(off, shf);
    tot = block_sum_f(tot, shf);
    if (tid == 0) s_done = (off <= kJacobiTol * tot) ? 1 : 0;
    __syncthreads();
    if (s_done) break;
    for (int r = 0; r < n - 1; ++r) {
      if (tid < n / 2) {
        int p, q;
        pair_of(r, tid, n, p, q);
        float c = 1.f, s = 0.f;
        if (q < k) {
          const float apq = Af[p][q];
          if (apq != 0.f) {
            const float theta = (Af[q][q] - Af[p][p]) / (2.f * apq);
            const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
            c = rsqrtf(t * t + 1.f);
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
      for (int w = tid; w < (n / 2) * k; w += kEx) {
        const int t = w / k, col = w % k;
        const int p = rp[t], q = rq[t];
        if (q < k) {
          const float c = rc[t], s = rs[t];
          const float ap = Af[p][col], aq = Af[q][col];
          Af[p][col] = c * ap - s * aq;
          Af[q][col] = s * ap + c * aq;
        }
      }
      __syncthreads();
      // A <- A J and V <- V J  (columns p, q of every pair)
      for (int w = tid; w < (n / 2) * k; w += kEx) {
        const int t = w / k, row = w % k;
        const int p = rp[t], q = rq[t];
        if (q < k) {
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
  for (int w = tid; w < k * k; w += kEx) {
    const int i = w / k, j = w % k;
    X[i][j] = (double)Vf[i][j];
  }
  float tnorm2 = 0.f;
  for (int i = tid; i < k; i += kEx) {
    tnorm2 += (float)al[i] * (float)al[i];
    if (i + 1 < k) tnorm2 += 2.f * (float)be[i] * (float)be[i];
  }
  const double tnorm = (double)sqrtf(block_sum_f(tnorm2, shf));   // ||T||_F (also syncs X)
  for (int it = 0; it < kRefineIters; ++it) {
    // W = T X
    for (int w = tid; w < k * k; w += kEx) {
      const int i = w / k, e = w % k;
      double v = al[i] * X[i][e];
      if (i > 0) v = fma(be[i - 1], X[i - 1][e], v);
      if (i + 1 < k) v = fma(be[i], X[i + 1][e], v);
      W[i][e] = v;
    }
    __syncthreads();
    // R = I - X^T X,  S = X^T T X  (two independent FMA chains each, for ILP)
    for (int w = tid; w < k * k; w += kEx) {
      const int a = w / k, b = w % k;
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
      R[a][b] = ((a == b) ? 1.0 : 0.0) - (r0 + r1);
      S[a][b] = s0 + s1;
    }
    __syncthreads();
    if (tid < k) lam[tid] = fast_div(S[tid][tid], 1.0 - R[tid][tid]);
    __syncthreads();
    float sd2 = 0.f, r2 = 0.f;
    for (int w = tid; w < k * k; w += kEx) {
      const int a = w / k, b = w % k;
      const float d = (float)(S[a][b] - ((a == b) ? lam[a] : 0.0));
      const float rr = (float)R[a][b];
      sd2 += d * d;
      r2 += rr * rr;
    }
    const float sdn = sqrtf(block_sum_f(sd2, shf));
    const float rn = sqrtf(block_sum_f(r2, shf));
    const double delta = 2.0 * ((double)sdn + tnorm * (double)rn);
    // E (stored in W)
    for (int w = tid; w < k * k; w += kEx) {
      const int a = w / k, b = w % k;
      double e;
      const double gap = lam[b] - lam[a];
      if (a == b || fabs(gap) <= delta) e = 0.5 * R[a][b];
      else e = fast_div(S[a][b] + lam[b] * R[a][b], gap);
      W[a][b] = e;
    }
    __syncthreads();
    // X <- X + X E   (new X into S, then copy)
    for (int w = tid; w < k * k; w += kEx) {
      const int i = w / k, b = w % k;
      double v0 = X[i][b], v1 = 0.0;
      int a = 0;
      for (; a + 1 < k; a += 2) {
        v0 = fma(X[i][a], W[a][b], v0);
        v1 = fma(X[i][a + 1], W[a + 1][b], v1);
      }
      if (a < k) v0 = fma(X[i][a], W[a][b], v0);
      S[i][b] = v0 + v1;
    }
    __syncthreads();
    for (int w = tid; w < k * k; w += kEx) {
      const int i = w / k, b = w % k;
      X[i][b] = S[i][b];
    }
    __syncthreads();
  }

  // ---- c_i = sum_e X_ie X_0e exp(-i lambda_e dt) --------------------------
  if (tid < k) {
    double sn, cs;
    sincos(lam[tid] * dt, &sn, &cs);
    W[0][tid] = X[0][tid] * cs;    // Re
    W[1][tid] = -X[0][tid] * sn;   // Im
  }
  __syncthreads();
  if (tid < KP) {
    double2 c = make_double2(0.0, 0.0);
    if (tid < k) {
      for (int e = 0; e < k; ++e) {
        c.x = fma(X[tid][e], W[0][e], c.x);
        c.y = fma(X[tid][e], W[1][e], c.y);
      }
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

cudaError_t launch_lanczos_expm(int m, double dt, LanczosScalars *ls, cudaStream_t st) {
  lanczos_expm_kernel<<<1, kEx, 0, st>>>(m, dt, ls);
  return cudaGetLastError();
}

}  // namespace tdse_dev
