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

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum_d(double v, double *sh) {
  const int tid = threadIdx.x;
  v = warp_sum_d(v);
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    double s = (tid < kEx / 32) ? sh[tid] : 0.0;
    s = warp_sum_d(s);
    if (tid == 0) sh[kEx / 32] = s;
  }
  __syncthreads();
  const double r = sh[kEx / 32];
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

__global__ void __launch_bounds__(kEx) lanczos_expm_kernel(int m, double dt, LanczosScalars *ls) {
  __shared__ double al[KP], be[KP];
  __shared__ float Af[KP][KP + 1];
  __shared__ float Vf[KP][KP + 1];
  __shared__ float rc[KP / 2], rs[KP / 2];
  __shared__ int rp[KP / 2], rq[KP / 2];
  __shared__ double X[KP][KP + 1], W[KP][KP + 1], R[KP][KP + 1], S[KP][KP + 1];
  __shared__ double lam[KP];
  __shared__ double sh[kEx / 32 + 1];
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
    double off = 0.0, tot = 0.0;
    for (int w = tid; w < k * k; w += kEx) {
      const int i = w / k, j = w % k;
      const double v = (double)Af[i][j];
      tot += v * v;
      if (i != j) off += v * v;
    }
    off = block_sum_d(off, sh);
    tot = block_sum_d(tot, sh);
    if (tid == 0) s_done = (off <= 1e-14 * tot) ? 1 : 0;
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
  double tnorm2 = 0.0;
  for (int i = tid; i < k; i += kEx) {
    tnorm2 += al[i] * al[i];
    if (i + 1 < k) tnorm2 += 2.0 * be[i] * be[i];
  }
  const double tnorm = sqrt(block_sum_d(tnorm2, sh));   // ||T||_F (also syncs X)
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
    // R = I - X^T X,  S = X^T T X
    for (int w = tid; w < k * k; w += kEx) {
      const int a = w / k, b = w % k;
      double r = 0.0, s = 0.0;
      for (int i = 0; i < k; ++i) {
        r = fma(X[i][a], X[i][b], r);
        s = fma(X[i][a], W[i][b], s);
      }
      R[a][b] = ((a == b) ? 1.0 : 0.0) - r;
      S[a][b] = s;
    }
    __syncthreads();
    if (tid < k) lam[tid] = S[tid][tid] / (1.0 - R[tid][tid]);
    __syncthreads();
    double sd2 = 0.0, r2 = 0.0;
    for (int w = tid; w < k * k; w += kEx) {
      const int a = w / k, b = w % k;
      const double d = S[a][b] - ((a == b) ? lam[a] : 0.0);
      sd2 += d * d;
      r2 += R[a][b] * R[a][b];
    }
    const double delta = 2.0 * (sqrt(block_sum_d(sd2, sh)) + tnorm * sqrt(block_sum_d(r2, sh)));
    // E (stored in W)
    for (int w = tid; w < k * k; w += kEx) {
      const int a = w / k, b = w % k;
      double e;
      const double gap = lam[b] - lam[a];
      if (a == b || fabs(gap) <= delta) e = 0.5 * R[a][b];
      else e = (S[a][b] + lam[b] * R[a][b]) / gap;
      W[a][b] = e;
    }
    __syncthreads();
    // X <- X + X E   (new X into S, then copy)
    for (int w = tid; w < k * k; w += kEx) {
      const int i = w / k, b = w % k;
      double v = X[i][b];
      for (int a = 0; a < k; ++a) v = fma(X[i][a], W[a][b], v);
      S[i][b] = v;
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
