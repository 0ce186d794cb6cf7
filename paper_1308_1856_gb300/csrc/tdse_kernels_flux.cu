// Dipole moments and the flux through a sphere (arXiv 1308.1856, Sec. 4).
//
// dipole_moments_kernel: <z>, d<z>/dt and d^2<z>/dt^2 of the state (m = 0):
//   <z>     = 2 sum_l kappa_{l+1} dr sum_j r_j Re(f_l^* f_{l+1})             (Eq. (Dipole))
//   <zdot>  = 2 sum_l kappa_{l+1} dr sum_j Im(f_{l+1}^* (D1 f_l - (l+1)/r_j f_l))
//             [+ (A/c) norm in the velocity gauge]                          (Eq. (DipoleVelocity))
//   <zddot> = -E norm - 2 Z sum_l kappa_{l+1} dr sum_j Re(f_l^* f_{l+1}) / r_j^2 (Eq. (DipoleAccel))
// D1 is the first-derivative formula of the velocity gauge.  The factor 2 of
// <zdot> (absent from the printed Eq. (DipoleVelocity)) is the one Ehrenfest's
// theorem d<z>/dt = <zdot> needs; <zdot> is the kinetic momentum.  Grid:
// (blocks per row, L + 1) blocks; block (x, l) sums its share of row l (and of
// the pair (l, l+1)); the last block to arrive adds the per-block partials in
// a fixed order, so the result does not depend on timing.
//
// flux_kernel: one block.  At the grid point j_b nearest r_b it forms
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
constexpr int kDipQ = 4;            // norm, r Re(f_l^* f_{l+1}), Im(...), Re(...)/r^2
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
  // first derivative of row l at i: 5-point [-f+2 + 8 f+1 - 8 f-1 + f-2] d1c,
  // 3-point [f+1 - f-1] d1c
  __device__ __forceinline__ double2 d1(int l, int i, int stencil, double d1c) const {
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
    return make_double2(__dmul_rn(s.x, d1c), __dmul_rn(s.y, d1c));
  }
};

__global__ void __launch_bounds__(kDipThreads)
    dipole_moments_kernel(RowReader rd, const double *__restrict__ rj, const double *__restrict__ kappa,
                          int L, int stencil, double dr, double d1c, double E, double ac, double Z,
                          int coulomb, double *partials, unsigned *ticket, double *out) {
  __shared__ double sh[kDipThreads / 32 + 1];
  __shared__ unsigned s_last;
  const int l = blockIdx.y;
  const int nbx = gridDim.x;
  const int N = rd.N;
  double q[kDipQ] = {0.0, 0.0, 0.0, 0.0};
  for (int i = blockIdx.x * kDipThreads + threadIdx.x; i < N; i += nbx * kDipThreads) {
    const double2 a = rd.psi[(size_t)l * N + i];
    q[0] = __fma_rn(a.x, a.x, __fma_rn(a.y, a.y, q[0]));
    if (l < L) {
      const double2 b = rd.psi[(size_t)(l + 1) * N + i];
      const double r = rj[i];
      const double rinv = 1.0 / r;
      const double re = __fma_rn(a.x, b.x, __dmul_rn(a.y, b.y));      // Re(conj(a) b)
      const double2 d = rd.d1(l, i, stencil, d1c);
      const double cl = __dmul_rn((double)(l + 1), rinv);
      const double2 w = make_double2(__fma_rn(-cl, a.x, d.x), __fma_rn(-cl, a.y, d.y));
      q[1] = __fma_rn(r, re, q[1]);
      q[2] = __fma_rn(b.x, w.y, __fma_rn(-b.y, w.x, q[2]));           // Im(conj(b) w)
      q[3] = __fma_rn(__dmul_rn(rinv, rinv), re, q[3]);
    }
  }
  const size_t nb = (size_t)nbx * (L + 1);
  const size_t bid = (size_t)l * nbx + blockIdx.x;
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
  // last block: per-row sums in block order, weighted by the row's kappa
  double np = 0.0, zp = 0.0, vp = 0.0, fp = 0.0;
  for (int row = threadIdx.x; row <= L; row += kDipThreads) {
    double p[kDipQ] = {0.0, 0.0, 0.0, 0.0};
    for (int bx = 0; bx < nbx; ++bx)
      for (int k = 0; k < kDipQ; ++k) p[k] += __ldcg(&partials[(size_t)k * nb + (size_t)row * nbx + bx]);
    np += p[0];
    if (row < L) {
      const double w = 2.0 * kappa[row + 1] * dr;
      zp = __fma_rn(w, p[1], zp);
      vp = __fma_rn(w, p[2], vp);
      fp = __fma_rn(w, p[3], fp);
    }
  }
  const double norm = dr * block_sum(np, sh);
  const double z = block_sum(zp, sh);
  const double v = block_sum(vp, sh);
  const double f = block_sum(fp, sh);
  if (threadIdx.x == 0) {
    out[0] = z;
    out[1] = __fma_rn(ac, norm, v);
    out[2] = coulomb ? __fma_rn(-E, norm, -Z * f) : __longlong_as_double(0x7ff8000000000000LL);
    *ticket = 0u;
  }
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
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int l = 0; l <= L; ++l) tot = __fma_rn(fb[l].x, db[l].y, __fma_rn(-fb[l].y, db[l].x, tot));
    if (ac != 0.0)
      for (int l = 0; l < L; ++l)
        tot = __fma_rn(2.0 * ac * kappa[l + 1], __fma_rn(fb[l].x, fb[l + 1].x, __dmul_rn(fb[l].y, fb[l + 1].y)), tot);
    if (!init) state[1] = __fma_rn(half_dt, __dadd_rn(state[0], tot), state[1]);
    else state[1] = 0.0;
    state[0] = tot;
  }
  for (int k = threadIdx.x; k < ntheta; k += kFluxThreads) {
    double2 S = make_double2(0.0, 0.0), P = make_double2(0.0, 0.0);
    for (int l = 0; l <= L; ++l) {
      const double y = ytab[(size_t)l * ntheta + k];
      S.x = __fma_rn(y, fb[l].x, S.x);
      S.y = __fma_rn(y, fb[l].y, S.y);
      P.x = __fma_rn(y, db[l].x, P.x);
      P.y = __fma_rn(y, db[l].y, P.y);
    }
    double dens = __fma_rn(S.x, P.y, -__dmul_rn(S.y, P.x));
    if (ac != 0.0) dens = __fma_rn(ac * cos_theta[k], __fma_rn(S.x, S.x, __dmul_rn(S.y, S.y)), dens);
    double *now = state + 2, *acc = state + 2 + ntheta;
    if (!init) acc[k] = __fma_rn(half_dt, __dadd_rn(now[k], dens), acc[k]);
    else acc[k] = 0.0;
    now[k] = dens;
  }
}

}  // namespace

int dipole_blocks(const Geometry &g) {
  const int per_row = (g.N + kDipThreads - 1) / kDipThreads;
  return per_row < 8 ? per_row : 8;
}

cudaError_t launch_dipole_moments(const Geometry &g, const OperatorView &op, const double2 *psi,
                                  int ghost, double E, double ac, double Z, bool coulomb,
                                  double *partials, unsigned *ticket, double *out, cudaStream_t st) {
  const int nbx = dipole_blocks(g);
  const dim3 grid(nbx, g.L + 1);
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
  flux_kernel<<<1, kFluxThreads, flux_shared_bytes(g), st>>>(rd, ib, g.L, g.stencil, d1c, ac, op.kappa, ytab,
                                                             cos_theta, ntheta, 0.5 * dt, init ? 1 : 0, state);
  return cudaGetLastError();
}

}  // namespace tdse_dev
