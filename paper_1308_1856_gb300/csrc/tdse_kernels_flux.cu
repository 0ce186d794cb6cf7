// Dipole moments and the flux through a sphere (arXiv 1308.1856, Sec. 4).
//
// dipole_moments_kernel: <z>, d<z>/dt and d^2<z>/dt^2 of the state (m = 0):
//   <z>     = 2 sum_l kappa_{l+1} dr sum_j r_j Re(f_l^* f_{l+1})             (Eq. (Dipole))
//   <zdot>  = 2 sum_l kappa_{l+1} dr sum_j Im(f_{l+1}^* (D1 f_l - (l+1)/r_j f_l))
//             [+ (A/c) norm in the velocity gauge]                          (Eq. (DipoleVelocity))
//   <zddot> = -E norm - 2 Z sum_l kappa_{l+1} dr sum_j Re(f_l^* f_{l+1}) / r_j^2 (Eq. (DipoleAccel))
// D1 is the first-derivative formula of the velocity gauge.  The factor 2 of
// <zdot> (absent from the printed Eq. (DipoleVelocity)) is the one Ehrenfest's
// theorem d<z>/dt = <zdot> needs; <zdot> is the kinetic momentum.  The last
// block to arrive adds the per-block partials in a fixed order, so the result
// does not depend on timing.
//
// flux_kernel: at the grid point j_b nearest r_b it forms
//   total  = sum_l Im(f_l^* D1 f_l) [+ 2 (A/c) sum_l kappa_{l+1} Re(f_l^* f_{l+1})]
//   dens_k = Im(S_k^* P_k) [+ (A/c) cos(theta_k) |S_k|^2],
//   S_k = sum_l Y_l0(theta_k) f_l(r_b),  P_k = sum_l Y_l0(theta_k) (D1 f_l)(r_b),
// r_b^2 times the radial current integrated over the sphere and per unit
// solid angle (Eqs. (flux), (pad), (yield); outward positive, the sign the
// continuity equation fixes), and advances their time integrals by the
// trapezoid rule: acc += (dt/2)(previous + current).
#include <cuda_runtime.h>

#include "tdse_device_common.cuh"
#include "tdse_internal.cuh"

namespace tdse_dev {

namespace {

using namespace common;

constexpr int kDipThreads = 256;
constexpr int kDipQ = 4;            // norm and the weighted <z>, <zdot>, <zddot> sums
constexpr int kDipRows = 4;         // partial waves per thread of the dipole kernel
constexpr int kFluxThreads = 256;

struct RowReader {
  const double2 *psi;
  int N, ghost;
  // f_{l,i}, i 0-based; zero outside the box, f_{l,-2} = -f_{l,0} with the odd ghost
  __device__ __forceinline__ double2 at(int l, int i) const {
    if (i >= 0 && i < N) return psi[(size_t)l * N + i];
    if (ghost && i == -2) {
      const double2 v = psi[(size_t)l * N];
      return make_double2(-v.x, -v.y);
    }
    return make_double2(0.0, 0.0);
  }
  // first derivative of row l at i without its scale: 5-point
  // -f+2 + 8 f+1 - 8 f-1 + f-2 (scale 1/(12 dr)), 3-point f+1 - f-1 (1/(2 dr))
  __device__ __forceinline__ double2 d1raw(int l, int i, int stencil) const {
    const double2 p1 = at(l, i + 1), m1 = at(l, i - 1);
    double2 s;
    if (stencil == 5) {
      const double2 p2 = at(l, i + 2), m2 = at(l, i - 2);
      s.x = __dadd_rn(__fma_rn(8.0, __dsub_rn(p1.x, m1.x), m2.x), -p2.x);
      s.y = __dadd_rn(__fma_rn(8.0, __dsub_rn(p1.y, m1.y), m2.y), -p2.y);
    } else {
      s.x = __dsub_rn(p1.x, m1.x);
      s.y = __dsub_rn(p1.y, m1.y);
    }
    return s;
  }
  __device__ __forceinline__ double2 d1(int l, int i, int stencil, double d1c) const {
    const double2 s = d1raw(l, i, stencil);
    return make_double2(__dmul_rn(s.x, d1c), __dmul_rn(s.y, d1c));
  }
};

// One thread per (radial index i, chunk of kDipRows partial waves): the
// thread walks l upwards keeping f_{l+1,i} for the next row, so the state is
// read once (plus the first-derivative neighbours, which the neighbouring
// lanes load too).  Per point it accumulates only row-weighted sums
// (w_l = 2 kappa_{l+1} dr):
//   S_re = sum_l w_l Re(f_l^* f_{l+1}),  S_d = sum_l w_l Im(f_{l+1}^* D1raw f_l),
//   S_c  = sum_l w_l (l+1) Im(f_{l+1}^* f_l),  S_n = sum_l |f_l|^2,
// and the radial factors r, 1/r^2, 1/r and the derivative scale are applied
// once per thread: <z> gets r S_re, <zddot> 1/r^2 S_re, <zdot> d1c S_d - S_c / r.
// (The FP64 pipe issues at 2 lanes/clock/SM, so the per-point instruction
// count sets this kernel's time.)  Each block publishes one partial per
// quantity and the last block adds them in a fixed order.
__global__ void __launch_bounds__(kDipThreads)
    dipole_moments_kernel(RowReader rd, const double *__restrict__ rj, const double *__restrict__ kappa,
                          int L, int stencil, double dr, double d1c, double E, double ac, double Z,
                          int coulomb, double *partials, unsigned *ticket, double *out) {
  __shared__ double sh[kDipThreads / 32 + 1];
  __shared__ double wrow[kDipRows], wrow1[kDipRows];
  __shared__ unsigned s_last;
  const int N = rd.N;
  const int i = blockIdx.x * kDipThreads + threadIdx.x;
  const int l0 = blockIdx.y * kDipRows;
  const int l1 = min(l0 + kDipRows, L + 1);
  if (threadIdx.x < kDipRows) {
    const int l = l0 + threadIdx.x;
    const double w = (l < L) ? 2.0 * kappa[l + 1] * dr : 0.0;
    wrow[threadIdx.x] = w;
    wrow1[threadIdx.x] = (double)(l + 1) * w;
  }
  __syncthreads();
  double q[kDipQ] = {0.0, 0.0, 0.0, 0.0};
  if (i < N) {
    double sn = 0.0, sre = 0.0, sd = 0.0, sc = 0.0;
    double2 a = rd.psi[(size_t)l0 * N + i];
    for (int l = l0; l < l1; ++l) {
      sn = __fma_rn(a.x, a.x, __fma_rn(a.y, a.y, sn));
      if (l < L) {
        const double2 b = rd.psi[(size_t)(l + 1) * N + i];
        const double w = wrow[l - l0], w1 = wrow1[l - l0];
        const double2 d = rd.d1raw(l, i, stencil);
        sre = __fma_rn(w, __fma_rn(a.x, b.x, __dmul_rn(a.y, b.y)), sre);       // Re(conj(a) b)
        sd = __fma_rn(w, __fma_rn(b.x, d.y, -__dmul_rn(b.y, d.x)), sd);       // Im(conj(b) d)
        sc = __fma_rn(w1, __fma_rn(b.x, a.y, -__dmul_rn(b.y, a.x)), sc);      // Im(conj(b) a)
        a = b;
      }
    }
    const double r = rj[i];
    const double rinv = 1.0 / r;
    q[0] = sn;
    q[1] = __dmul_rn(r, sre);
    q[2] = __fma_rn(d1c, sd, -__dmul_rn(rinv, sc));
    q[3] = __dmul_rn(__dmul_rn(rinv, rinv), sre);
  }
  const unsigned nb = gridDim.x * gridDim.y;
  const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
  for (int k = 0; k < kDipQ; ++k) {
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
  // last block: thread t adds the partials of blocks t, t + blockDim, ... and
  // a fixed tree adds the threads' sums (every load is issued before the adds)
  double tot[kDipQ];
  for (int k = 0; k < kDipQ; ++k) {
    double v = 0.0;
    for (unsigned b = threadIdx.x; b < nb; b += kDipThreads) v += __ldcg(&partials[(size_t)k * nb + b]);
    tot[k] = block_sum(v, sh);
  }
  if (threadIdx.x == 0) {
    const double norm = dr * tot[0];
    out[0] = tot[1];
    out[1] = __fma_rn(ac, norm, tot[2]);
    out[2] = coulomb ? __fma_rn(-E, norm, -Z * tot[3]) : __longlong_as_double(0x7ff8000000000000LL);
    *ticket = 0u;
  }
}

// Flux: one warp per angle (8 per block); the lanes split the partial waves
// and a fixed butterfly adds their shares.  Warp 0 of block 0 first forms the
// total.  Every block stages f_l(r_b) and (D1 f_l)(r_b) in shared memory.
__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kFluxThreads)
    flux_kernel(RowReader rd, int ib, int L, int stencil, double d1c, double ac,
                const double *__restrict__ kappa, const double *__restrict__ ytab,
                const double *__restrict__ cos_theta, int ntheta, double half_dt, int init,
                double *state) {
  // state: [0] total now, [1] total integral, [2 .. 2+nt) density now, [2+nt .. 2+2nt) density integral
  extern __shared__ double2 fsh[];
  double2 *fb = fsh, *db = fsh + (L + 1);
  for (int l = threadIdx.x; l <= L; l += kFluxThreads) {
    fb[l] = rd.at(l, ib);
    db[l] = rd.d1(l, ib, stencil, d1c);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (blockIdx.x == 0 && warp == 0) {
    double tot = 0.0;
    for (int l = lane; l <= L; l += 32) {
      tot = __fma_rn(fb[l].x, db[l].y, __fma_rn(-fb[l].y, db[l].x, tot));
      if (ac != 0.0 && l < L)
        tot = __fma_rn(2.0 * ac * kappa[l + 1], __fma_rn(fb[l].x, fb[l + 1].x, __dmul_rn(fb[l].y, fb[l + 1].y)), tot);
    }
    tot = warp_allsum(tot);
    if (lane == 0) {
      if (!init) state[1] = __fma_rn(half_dt, __dadd_rn(state[0], tot), state[1]);
      else state[1] = 0.0;
      state[0] = tot;
    }
  }
  const int k = blockIdx.x * (kFluxThreads / 32) + warp;
  if (k >= ntheta) return;
  const double *yk = ytab + (size_t)k * (L + 1);
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
    if (ac != 0.0) dens = __fma_rn(ac * cos_theta[k], __fma_rn(sx, sx, __dmul_rn(sy, sy)), dens);
    double *now = state + 2, *acc = state + 2 + ntheta;
    if (!init) acc[k] = __fma_rn(half_dt, __dadd_rn(now[k], dens), acc[k]);
    else acc[k] = 0.0;
    now[k] = dens;
  }
}

}  // namespace

int dipole_blocks(const Geometry &g) {
  return ((g.N + kDipThreads - 1) / kDipThreads) * ((g.L + kDipRows) / kDipRows);
}

cudaError_t launch_dipole_moments(const Geometry &g, const OperatorView &op, const double2 *psi,
                                  int ghost, double E, double ac, double Z, bool coulomb,
                                  double *partials, unsigned *ticket, double *out, cudaStream_t st) {
  const dim3 grid((g.N + kDipThreads - 1) / kDipThreads, (g.L + kDipRows) / kDipRows);
  const RowReader rd{psi, g.N, ghost};
  const double d1c = (g.stencil == 5) ? 1.0 / (12.0 * g.dr) : 1.0 / (2.0 * g.dr);
  dipole_moments_kernel<<<grid, kDipThreads, 0, st>>>(rd, op.rj, op.kappa, g.L, g.stencil, g.dr, d1c, E, ac,
                                                      Z, coulomb ? 1 : 0, partials, ticket, out);
  return cudaGetLastError();
}

size_t flux_shared_bytes(const Geometry &g) { return sizeof(double2) * 2 * (size_t)(g.L + 1); }

cudaError_t launch_flux(const Geometry &g, const OperatorView &op, const double2 *psi, int ghost,
                        int ib, double ac, const double *ytab, const double *cos_theta, int ntheta,
                        double dt, bool init, double *state, cudaStream_t st) {
  const RowReader rd{psi, g.N, ghost};
  const double d1c = (g.stencil == 5) ? 1.0 / (12.0 * g.dr) : 1.0 / (2.0 * g.dr);
  const int per_block = kFluxThreads / 32;
  const unsigned blocks = ntheta > 0 ? (unsigned)((ntheta + per_block - 1) / per_block) : 1u;
  flux_kernel<<<blocks, kFluxThreads, flux_shared_bytes(g), st>>>(rd, ib, g.L, g.stencil, d1c, ac, op.kappa, ytab,
                                                                  cos_theta, ntheta, 0.5 * dt, init ? 1 : 0, state);
  return cudaGetLastError();
}

}  // namespace tdse_dev
