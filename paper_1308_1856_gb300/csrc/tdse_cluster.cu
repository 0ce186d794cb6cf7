// Small grids in one launch: every step of a run inside one thread-block
// cluster, with the state and the work vectors resident in shared memory.
//
// A grid of a few thousand points (the small configuration: N = 500,
// lmax = 4, 2,500 points, 40 KB per vector) is a few microseconds of FP64
// arithmetic per step.  Launched as one kernel per stage (Taylor, RK4) or two
// per Lanczos iteration, every launch pays its launch latency and a grid-wide
// reduction, and the step is latency bound.  Here one cluster of C CTAs
// (C <= 16, one per SM, 256 threads each) runs the whole propagation of
// Sec. 5 ("Taylor.c", "RungeKutta.c", "Lanczos.c" of arXiv 1308.1856):
//   - CTA r owns the radial columns [r W, min((r+1) W, N)) of every partial
//     wave; its slice of psi, of the diagonal table and of every work vector
//     stays in its shared memory for the whole run;
//   - the 3- or 5-point stencil of Eq. (h_matrix) reads the one or two
//     columns beyond the slice from the neighbouring CTA's shared memory
//     (distributed shared memory); the l-neighbour rows are in the slice;
//   - a cluster barrier separates the stages: each stage reads the halo of
//     the vector the previous stage wrote;
//   - a grid-wide sum (the Lanczos dot products and norms) is every warp's
//     shuffle-tree sum, a cluster barrier, and the C x 8 warp sums added in
//     one fixed order by warp 0 of every CTA, so that every CTA holds the
//     same bits (cluster_sum);
//   - every CTA forms the small exponential of the Lanczos step itself from
//     those identical scalars, so no broadcast is needed.
// The per-point arithmetic of Taylor and RK4 is that of the multi-launch
// kernels (tdse_kernels_fp64.cu), so either path gives bitwise the same state;
// the field couplings kappa_l E r_j of a Taylor or Lanczos step are formed
// once per step into a table, with the walker's roundings.  Lanczos applies
// the unscaled operator and then sigma_j (the multi-launch kernels fold
// sigma_j into the coefficients), and associates its grid sums differently:
// it agrees with that path to rounding.
// The only waits are cluster barriers (hardware), reached the same number of
// times by every CTA: the control flow is uniform over the cluster.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "tdse_device_common.cuh"
#include "tdse_internal.cuh"
#include "tdse_small_expm.cuh"

namespace cg = cooperative_groups;

namespace tdse_dev {

namespace {

using common::warp_sum;

constexpr int kCT = 256;   // threads per CTA
static_assert(kCT == kEx, "the small exponential body runs on the whole CTA");
constexpr int kMaxCluster = 16;

template <bool B>
struct BoolC {
  static constexpr bool value = B;
};

struct SmallDev {
  double2 *psi;
  const double *diag, *rj, *kappa, *mask;
  const double *etab;     // per step: the mid-step field (Taylor, Lanczos) or the
                          // three stage fields t_n, t_n + dt/2, t_n + dt (RK4)
  LanczosScalars *ls;
  Reduction *red;
  int *status;
  int N, L, W, mask_start, order, nsteps;
  double c1, c2, dt;
};

// This CTA's slice in shared memory.
struct Slab {
  double2 *v;              // NV vectors of VS = (L+1) W complex values, [vec][l][jl]
  double *diag;            // [l][jl]
  double *rj, *mask;       // [jl]
  double *kappa;           // [0, L+1]
  double *ea;              // [0, L+1][jl]: kappa_l E r_j of the current step
  int VS, W, Wc, j0, N, L;
  int rank;
};

// Column q (local index, may fall one or two columns outside the slice) of
// the row starting at `row`: zero beyond the box, else from this CTA or the
// neighbour that owns it.  The layout is the same in every CTA, so the
// neighbour's copy of a row sits at the same offset of its shared memory.
__device__ __forceinline__ double2 col(const cg::cluster_group &cl, const Slab &s, const double2 *row, int q) {
  const int j = s.j0 + q;
  if (j < 0 || j >= s.N) return make_double2(0.0, 0.0);
  if (q < 0) return *cl.map_shared_rank(row + (q + s.W), s.rank - 1);
  if (q >= s.W) return *cl.map_shared_rank(row + (q - s.W), s.rank + 1);
  return row[q];
}

// (H x) at (l, jl), length gauge, given the diagonal d and the two coupling
// coefficients a_cur (to l - 1) and a_next (to l + 1) of the point: the FP64
// operations of the multi-launch walker (h_point / walk_rows) in its order.
template <int ST>
__device__ __forceinline__ double2 h_core(const cg::cluster_group &cl, const Slab &s, const double2 *x, int l,
                                          int jl, double c1, double c2, double d, double a_cur, double a_next) {
  const double2 z = make_double2(0.0, 0.0);
  const double2 *row = x + l * s.W;
  const double2 cur = row[jl];
  const double2 prev = (l > 0) ? row[jl - s.W] : z;
  const double2 next = (l < s.L) ? row[jl + s.W] : z;
  const double2 m1 = col(cl, s, row, jl - 1), p1 = col(cl, s, row, jl + 1);
  double tx = __dmul_rn(d, cur.x);
  double ty = __dmul_rn(d, cur.y);
  tx = __fma_rn(c1, __dadd_rn(m1.x, p1.x), tx);
  ty = __fma_rn(c1, __dadd_rn(m1.y, p1.y), ty);
  if (ST == 5) {
    const double2 m2 = col(cl, s, row, jl - 2), p2 = col(cl, s, row, jl + 2);
    tx = __fma_rn(c2, __dadd_rn(m2.x, p2.x), tx);
    ty = __fma_rn(c2, __dadd_rn(m2.y, p2.y), ty);
  }
  tx = __fma_rn(a_cur, prev.x, tx);
  ty = __fma_rn(a_cur, prev.y, ty);
  tx = __fma_rn(a_next, next.x, tx);
  ty = __fma_rn(a_next, next.y, ty);
  return make_double2(tx, ty);
}

// (H x) at (l, jl) in field E, every coefficient formed at the point.
template <int ST>
__device__ __forceinline__ double2 h_at(const cg::cluster_group &cl, const Slab &s, const double2 *x, int l,
                                        int jl, double c1, double c2, double E) {
  const double Er = __dmul_rn(E, s.rj[jl]);
  const double a_cur = __dmul_rn(s.kappa[l], Er);
  const double a_next = __dmul_rn(s.kappa[l + 1], Er);
  return h_core<ST>(cl, s, x, l, jl, c1, c2, s.diag[l * s.W + jl], a_cur, a_next);
}

// (H x) at (l, jl) with the coupling coefficients of the step taken from the
// table ea[l][jl] = kappa_l (E r_j), l = 0 .. L + 1 (filled by fill_coupling):
// the same values h_at forms point by point, without its three products.
template <int ST>
__device__ __forceinline__ double2 h_tab(const cg::cluster_group &cl, const Slab &s, const double2 *x, int l,
                                         int jl, double c1, double c2, const double *ea) {
  const int idx = l * s.W + jl;
  return h_core<ST>(cl, s, x, l, jl, c1, c2, s.diag[idx], ea[idx], ea[idx + s.W]);
}

// ea[l][jl] = kappa_l (E r_j) for l = 0 .. L + 1 and the slice's columns,
// in h_at's order of rounding.  Called by every thread of the CTA; the caller
// orders it against the table's readers with a CTA barrier.
__device__ __forceinline__ void fill_coupling(const Slab &s, double E) {
  const int n = (s.L + 2) * s.W;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int l = i / s.W, jl = i - l * s.W;
    if (jl < s.Wc) s.ea[i] = __dmul_rn(s.kappa[l], __dmul_rn(E, s.rj[jl]));
  }
}

// This thread's points of the slice: rows ty, ty + RP, ... and columns
// tx, tx + TW, ... (TW = min(W, 256) threads per row, RP = 256 / TW rows at
// a time).  The assignment is fixed, so every per-thread sum has a fixed order.
struct Lanes {
  int tx, ty, TW, RP;
};

template <typename F>
__device__ __forceinline__ void for_points(const Slab &s, const Lanes &ln, F &&f) {
  if (ln.ty >= ln.RP) return;
  for (int l = ln.ty; l <= s.L; l += ln.RP)
    for (int jl = ln.tx; jl < s.Wc; jl += ln.TW) f(l, jl, l * s.W + jl);
}

// Sum over the cluster, the same bits in every CTA.  Every warp publishes its
// shuffle-tree sum in one of two slot sets (alternating, so a set is
// rewritten only after a later cluster barrier, when every CTA has read it);
// after the cluster barrier warp 0 of every CTA adds the C x 8 warp sums in
// one fixed order (lane t: the sums t, t + 32, t + 64, t + 96 in pairs, then
// a shuffle tree), and thread 0 hands the total to `fin`, whose results the
// closing CTA barrier publishes.  Each FP64 instruction of this dependent
// chain holds the narrow FP64 pipe for a full pass, so the chain is kept
// short: 12 additions and one CTA barrier besides the cluster barrier.
constexpr int kWarps = kCT / 32;
static_assert(kMaxCluster * kWarps <= 128, "four warp sums per lane of warp 0");
struct ClusterSum {
  double *slot;    // [2][kWarps]
  int par;
};

template <typename Fin>
__device__ __forceinline__ void cluster_sum(const cg::cluster_group &cl, ClusterSum &cs, double v, int C,
                                            Fin &&fin) {
  const int lane = (int)threadIdx.x & 31, w = (int)threadIdx.x >> 5;
  double *set = cs.slot + cs.par * kWarps;
  v = warp_sum(v);
  if (lane == 0) set[w] = v;
  cl.sync();
  if (w == 0) {
    double p[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = lane + 32 * q;   // warp i % kWarps of CTA i / kWarps
      p[q] = (i < C * kWarps) ? *cl.map_shared_rank(set + (i % kWarps), i / kWarps) : 0.0;
    }
    const double t = warp_sum(__dadd_rn(__dadd_rn(p[0], p[1]), __dadd_rn(p[2], p[3])));
    if (lane == 0) fin(t);
  }
  __syncthreads();
  cs.par ^= 1;
}

// ||x|| and 1 / ||x|| from ||x||^2 with one reciprocal square root and one
// product (about half the dependent FP64 instructions of a square root and a
// division); 0 gives (0, 0), Inf or NaN gives (sqrt, 0).
__device__ __forceinline__ void norm_and_inverse(double s2, double &nrm, double &inv) {
  if (s2 > 0.0 && s2 <= 1.7976931348623157e308) {
    inv = rsqrt(s2);
    nrm = __dmul_rn(s2, inv);
  } else {
    nrm = sqrt(s2);
    inv = 0.0;
  }
}

// Sum of |x|^2 over this thread's points, in the order of the Lanczos combine.
__device__ __forceinline__ double norm_acc(const Slab &s, const Lanes &ln, const double2 *x) {
  double acc = 0.0;
  for_points(s, ln, [&](int, int, int idx) {
    const double2 v = x[idx];
    acc = __fma_rn(v.x, v.x, acc);
    acc = __fma_rn(v.y, v.y, acc);
  });
  return acc;
}

template <int ST, int METHOD>
__global__ void __launch_bounds__(kCT, 1) small_grid_kernel(SmallDev a) {
  const cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  __shared__ double s_slot[2 * kWarps];
  __shared__ LanczosScalars s_ls;
  __shared__ int s_bad;

  Slab s;
  s.rank = (int)cl.block_rank();
  const int C = (int)cl.num_blocks();
  s.N = a.N;
  s.L = a.L;
  s.W = a.W;
  s.j0 = s.rank * a.W;
  s.Wc = min(a.W, a.N - s.j0);
  s.VS = (a.L + 1) * a.W;
  const int NV = (METHOD == 0) ? 3 : (METHOD == 1 ? 4 : a.order + 1);
  s.v = reinterpret_cast<double2 *>(dyn_smem);
  s.diag = reinterpret_cast<double *>(s.v + (size_t)NV * s.VS);
  s.rj = s.diag + s.VS;
  s.mask = s.rj + s.W;
  s.kappa = s.mask + s.W;
  s.ea = s.kappa + (a.L + 2);
  auto V = [&](int k) { return s.v + (size_t)k * s.VS; };
  double2 *psi = V(0);

  Lanes ln;
  ln.TW = min(a.W, kCT);
  ln.RP = kCT / ln.TW;
  ln.tx = (int)threadIdx.x % ln.TW;
  ln.ty = (int)threadIdx.x / ln.TW;
  ClusterSum cs{s_slot, 0};
  const int N = a.N;

  // ---- this CTA's slice of psi and of the tables --------------------------
  for_points(s, ln, [&](int l, int jl, int idx) {
    const size_t g = (size_t)l * N + s.j0 + jl;
    psi[idx] = a.psi[g];
    s.diag[idx] = a.diag[g];
  });
  for (int jl = threadIdx.x; jl < s.Wc; jl += kCT) {
    s.rj[jl] = a.rj[s.j0 + jl];
    s.mask[jl] = a.mask[s.j0 + jl];
  }
  for (int l = threadIdx.x; l <= a.L + 1; l += kCT) s.kappa[l] = a.kappa[l];
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  cl.sync();   // every CTA of the cluster runs and holds its slice

  if constexpr (METHOD == 0) {
    // ---- Taylor polynomial in Horner form (Eq. (Taylor)) ------------------
    // The field is that of the mid-step for every stage: the coupling table
    // is formed once per step.  Only the last stage carries the absorber, in
    // its own instantiation (no mask instructions in the others).
    const int P = a.order;
    auto stage = [&](auto fin, const double2 *vin, double2 *out, double sk) {
      for_points(s, ln, [&](int l, int jl, int idx) {
        const double2 t = h_tab<ST>(cl, s, vin, l, jl, a.c1, a.c2, s.ea);
        const double2 p = psi[idx];
        double2 o = make_double2(__fma_rn(sk, t.y, p.x), __fma_rn(-sk, t.x, p.y));
        if constexpr (decltype(fin)::value) {
          if (s.j0 + jl >= a.mask_start) {
            const double mv = s.mask[jl];
            o.x = __dmul_rn(mv, o.x);
            o.y = __dmul_rn(mv, o.y);
          }
        }
        out[idx] = o;
      });
    };
    for (int n = 0; n < a.nsteps; ++n) {
      fill_coupling(s, a.etab[n]);
      __syncthreads();
      const double2 *vin = psi;
      for (int k = P; k >= 1; --k) {
        const bool last = (k == 1);
        double2 *out = last ? ((P == 1) ? V(1) : psi) : V(1 + ((P - k) & 1));
        const double sk = a.dt / (double)k;
        if (last)
          stage(BoolC<true>{}, vin, out, sk);
        else
          stage(BoolC<false>{}, vin, out, sk);
        cl.sync();
        vin = out;
      }
      if (P == 1) {
        for_points(s, ln, [&](int, int, int idx) { psi[idx] = V(1)[idx]; });
        cl.sync();
      }
    }
  } else if constexpr (METHOD == 1) {
    // ---- classic RK4 (Eq. (RKDeriv)), stage fields t_n, t_n + dt/2, t_n + dt
    double2 *ga = V(1), *gb = V(2), *acc = V(3);
    const double an[4] = {0.5, 0.5, 1.0, 0.0};
    const double bw[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    for (int n = 0; n < a.nsteps; ++n) {
      const double Es[4] = {a.etab[3 * n], a.etab[3 * n + 1], a.etab[3 * n + 1], a.etab[3 * n + 2]};
      const double2 *gin[4] = {psi, ga, gb, ga};
      double2 *gout[4] = {ga, gb, ga, nullptr};
#pragma unroll 1
      for (int st = 0; st < 4; ++st) {
        const double ca = a.dt * an[st], cb = a.dt * bw[st];
        const double2 *accin = (st == 0) ? psi : acc;
        for_points(s, ln, [&](int l, int jl, int idx) {
          const double2 t = h_at<ST>(cl, s, gin[st], l, jl, a.c1, a.c2, Es[st]);
          const double2 ai = accin[idx];
          if (st < 3) {
            const double2 p = psi[idx];
            gout[st][idx] = make_double2(__fma_rn(ca, t.y, p.x), __fma_rn(-ca, t.x, p.y));
            acc[idx] = make_double2(__fma_rn(cb, t.y, ai.x), __fma_rn(-cb, t.x, ai.y));
          } else {
            double2 o = make_double2(__fma_rn(cb, t.y, ai.x), __fma_rn(-cb, t.x, ai.y));
            if (s.j0 + jl >= a.mask_start) {
              const double mv = s.mask[jl];
              o.x = __dmul_rn(mv, o.x);
              o.y = __dmul_rn(mv, o.y);
            }
            psi[idx] = o;
          }
        });
        cl.sync();
      }
    }
  } else {
    // ---- Lanczos (Appendix "Lanczos methods") with U_j = q_j / sigma_j ----
    // V(1) = z, V(1 + j) = U_j for j >= 1, U_0 = psi.
    const int m = a.order;
    double2 *z = V(1);
    auto U = [&](int j) { return j == 0 ? psi : V(1 + j); };
    cluster_sum(cl, cs, norm_acc(s, ln, psi), C, [&](double s2) {
      norm_and_inverse(s2, s_ls.psinorm, s_ls.sigma[0]);
      if (!isfinite(s2)) s_bad = 1;
    });
    for (int n = 0; n < a.nsteps; ++n) {
      // the step's coupling table; its last readers (the previous step's
      // final iteration) are behind the cluster barriers of its sums
      fill_coupling(s, a.etab[n]);
      __syncthreads();
      for (int j = 0; j < m; ++j) {
        // z = sigma_j H U_j - ratio_j U_{j-1};  alpha_j = sigma_j Re <U_j, z>
        // (H U_j from the unscaled operator and the step's table, then
        // scaled by sigma_j: fewer FP64 instructions per point than scaling
        // every coefficient)
        const double sig = s_ls.sigma[j];
        const double cprev = (j > 0) ? s_ls.ratio[j] : 0.0;
        const double2 *u = U(j);
        const double2 *up = (j > 0) ? U(j - 1) : nullptr;
        double acc = 0.0;
        for_points(s, ln, [&](int l, int jl, int idx) {
          const double2 t = h_tab<ST>(cl, s, u, l, jl, a.c1, a.c2, s.ea);
          double2 o;
          if (j > 0) {
            const double2 pv = up[idx];
            o.x = __fma_rn(sig, t.x, __dmul_rn(-cprev, pv.x));
            o.y = __fma_rn(sig, t.y, __dmul_rn(-cprev, pv.y));
          } else {
            o.x = __dmul_rn(sig, t.x);
            o.y = __dmul_rn(sig, t.y);
          }
          z[idx] = o;
          const double2 uc = u[idx];
          acc = __fma_rn(uc.x, o.x, acc);
          acc = __fma_rn(uc.y, o.y, acc);
        });
        cluster_sum(cl, cs, acc, C, [&](double sa) {
          s_ls.alpha[j] = sa * sig;
          s_ls.acoef[j] = -(sa * sig) * sig;
        });
        if (j + 1 < m) {
          // U_{j+1} = z - alpha_j sigma_j U_j;  beta_j = ||U_{j+1}||
          const double c = s_ls.acoef[j];
          double2 *un = U(j + 1);
          double acc0 = 0.0, acc1 = 0.0;
          for_points(s, ln, [&](int, int, int idx) {
            const double2 uc = u[idx], zz = z[idx];
            const double2 o = make_double2(__fma_rn(c, uc.x, zz.x), __fma_rn(c, uc.y, zz.y));
            un[idx] = o;
            acc0 = __fma_rn(o.x, o.x, acc0);
            acc1 = __fma_rn(o.y, o.y, acc1);
          });
          cluster_sum(cl, cs, acc0 + acc1, C, [&](double sb) {
            double beta, sn;
            norm_and_inverse(sb, beta, sn);
            s_ls.beta[j] = beta;
            s_ls.sigma[j + 1] = sn;
            s_ls.ratio[j + 1] = (sn > 0.0) ? s_ls.sigma[j] * beta : 0.0;
          });
        }
      }
      // c = exp(-i T dt) e_1, formed by every CTA from the same scalars
      expm_body(m, a.dt, &s_ls, false);
      __syncthreads();
      // psi_new = sum_{j<k} coef_j U_j, the mask, ||psi_new||^2
      const int k = s_ls.kdim;
      double acc = 0.0;
      for_points(s, ln, [&](int, int jl, int idx) {
        const double2 u0 = psi[idx];
        const double2 c0 = s_ls.coef[0];
        double ox = __fma_rn(c0.x, u0.x, __dmul_rn(-c0.y, u0.y));
        double oy = __fma_rn(c0.x, u0.y, __dmul_rn(c0.y, u0.x));
        for (int jj = 1; jj < k; ++jj) {
          const double2 uu = U(jj)[idx];
          const double2 c = s_ls.coef[jj];
          ox = __fma_rn(c.x, uu.x, ox);
          ox = __fma_rn(-c.y, uu.y, ox);
          oy = __fma_rn(c.x, uu.y, oy);
          oy = __fma_rn(c.y, uu.x, oy);
        }
        if (s.j0 + jl >= a.mask_start) {
          const double mv = s.mask[jl];
          ox = __dmul_rn(mv, ox);
          oy = __dmul_rn(mv, oy);
        }
        psi[idx] = make_double2(ox, oy);
        acc = __fma_rn(ox, ox, acc);
        acc = __fma_rn(oy, oy, acc);
      });
      cluster_sum(cl, cs, acc, C, [&](double s2) {
        norm_and_inverse(s2, s_ls.psinorm, s_ls.sigma[0]);
        if (!isfinite(s2)) s_bad = 1;
        if (s.rank == 0) a.red->normsq = s2;
      });
    }
    if (s.rank == 0 && threadIdx.x == 0) {
      a.ls->psinorm = s_ls.psinorm;
      a.ls->sigma[0] = s_ls.sigma[0];
    }
  }

  // ---- the slice back to psi; Inf/NaN in the state -> status word ---------
  int bad = 0;
  for_points(s, ln, [&](int l, int jl, int idx) {
    const double2 v = psi[idx];
    a.psi[(size_t)l * N + s.j0 + jl] = v;
    if (!isfinite(v.x) || !isfinite(v.y)) bad = 1;
  });
  bad = __syncthreads_or(bad) | s_bad;
  if (bad && threadIdx.x == 0) atomicOr(a.status, kStatusNonFinite);
  cl.sync();   // no CTA leaves while a neighbour may still read its shared memory
}

template <int ST, int METHOD>
cudaError_t launch_one(const SmallPlan &p, const SmallDev &d, cudaStream_t st) {
  auto kern = small_grid_kernel<ST, METHOD>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)p.ctas, 1, 1);
  cfg.blockDim = dim3(kCT, 1, 1);
  cfg.dynamicSmemBytes = p.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)p.ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, d);
}

// Raise the kernel's limits once (dynamic shared memory, 16-CTA clusters) and
// report whether a cluster of `ctas` CTAs with `smem` bytes each can be
// resident on this device.
template <int ST, int METHOD>
bool fits(int ctas, size_t smem) {
  auto kern = small_grid_kernel<ST, METHOD>;
  static bool configured = false;
  static int max_dyn = 0;
  if (!configured) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    max_dyn = optin - (int)fa.sharedSizeBytes;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      max_dyn = 0;
    }
    configured = true;
  }
  if (max_dyn <= 0 || smem > (size_t)max_dyn) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas, 1, 1);
  cfg.blockDim = dim3(kCT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return nclusters >= 1;
}

template <int ST>
bool fits_m(int method, int ctas, size_t smem) {
  if (method == TDSE_TAYLOR) return fits<ST, 0>(ctas, smem);
  if (method == TDSE_RK4) return fits<ST, 1>(ctas, smem);
  return fits<ST, 2>(ctas, smem);
}

}  // namespace

SmallPlan plan_small_grid(const Geometry &g, int method, int order) {
  SmallPlan p;
  if (g.gauge != 0 || g.N < 2 || g.L < 0) return p;
  if (method != TDSE_TAYLOR && method != TDSE_RK4 && method != TDSE_LANCZOS) return p;
  if (method == TDSE_LANCZOS && (order < 1 || order > kMaxKrylov)) return p;
  if (method == TDSE_TAYLOR && order < 1) return p;
  const int nv = (method == TDSE_TAYLOR) ? 3 : (method == TDSE_RK4 ? 4 : order + 1);
  for (int cmax = kMaxCluster; cmax >= 2; cmax /= 2) {
    int W = (g.N + cmax - 1) / cmax;
    if (W < 2) W = 2;
    const int C = (g.N + W - 1) / W;
    const size_t VS = (size_t)(g.L + 1) * W;
    size_t bytes = sizeof(double2) * nv * VS +
                   sizeof(double) * (VS + 2 * (size_t)W + (size_t)g.L + 2 + (size_t)(g.L + 2) * W);
    bytes = (bytes + 15) & ~(size_t)15;
    const bool ok = (g.stencil == 5) ? fits_m<5>(method, C, bytes) : fits_m<3>(method, C, bytes);
    if (ok) {
      p.ok = true;
      p.ctas = C;
      p.W = W;
      p.smem = bytes;
      return p;
    }
  }
  return p;
}

cudaError_t launch_small_grid(const SmallPlan &p, const Geometry &g, const OperatorView &op, int method,
                              int order, double dt, long nsteps, const double *etab, double2 *psi,
                              LanczosScalars *ls, Reduction *red, int *status, cudaStream_t st) {
  if (!p.ok || nsteps < 1 || nsteps > 0x7fffffffL) return cudaErrorInvalidValue;
  SmallDev d;
  d.psi = psi;
  d.diag = op.diag;
  d.rj = op.rj;
  d.kappa = op.kappa;
  d.mask = op.mask;
  d.etab = etab;
  d.ls = ls;
  d.red = red;
  d.status = status;
  d.N = g.N;
  d.L = g.L;
  d.W = p.W;
  d.mask_start = op.mask_start;
  d.order = order;
  d.nsteps = (int)nsteps;
  d.c1 = g.c1;
  d.c2 = g.c2;
  d.dt = dt;
  if (g.stencil == 5) {
    if (method == TDSE_TAYLOR) return launch_one<5, 0>(p, d, st);
    if (method == TDSE_RK4) return launch_one<5, 1>(p, d, st);
    return launch_one<5, 2>(p, d, st);
  }
  if (method == TDSE_TAYLOR) return launch_one<3, 0>(p, d, st);
  if (method == TDSE_RK4) return launch_one<3, 1>(p, d, st);
  return launch_one<3, 2>(p, d, st);
}

}  // namespace tdse_dev
