// Internal declarations shared by the CUDA translation units of libtdse.
//
// Device data layout (all in HBM, owned by the handle):
//   psi      double2[(L+1)*N]  state F, l-major (Sec. 2, the vector F of Eq. (h_matrix))
//   diag     double [(L+1)*N]  c0 + l(l+1)/(2 r_j^2) + V(r_j)  (+ odd-ghost fold at j = 1)
//   rj       double [N]        r_j
//   kappa    double [L+2]      kappa_0 = 0, kappa_l (l = 1..L), kappa_{L+1} = 0
//   mask     double [N]        absorber mask (1 inside r_a)
//   work     double2[nvec*G]   Taylor / RK / Krylov work vectors
//   red      reduction slots (block partials, tickets, scalars)
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

#include "../../include/tdse.h"

namespace tdse_dev {

// NVTX range over one ABI call (visible in Nsight timelines; free without a tool).
struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

constexpr int kMaxKrylov = TDSE_MAX_KRYLOV;
// Persistent grids use few, large blocks (2 x 16 warps per SM): every block
// ends with one same-address atomic for the grid reduction, and those
// serialise in L2, so the block count sets the length of the reduction tail.
constexpr int kBlockJ = 512;            // threads per block of the stencil kernels
constexpr int kStencilBlocksPerSM = 2;
constexpr int kElemThreads = 512;       // threads per block of the elementwise kernels
constexpr int kElemBlocksPerSM = 2;
constexpr int kMaxPartials = 16384;     // block partial slots of one grid reduction

// Scalars of one Lanczos step, resident in device memory.
struct LanczosScalars {
  double alpha[kMaxKrylov];      // alpha_j = <q_j, H q_j>
  double beta[kMaxKrylov];       // beta_j = ||w_j|| (beta[j] links q_j and q_{j+1})
  double sigma[kMaxKrylov + 1];  // sigma_j = 1 / ||U_j||  (U_0 = psi, U_j unnormalised)
  double ratio[kMaxKrylov + 1];  // ratio_j = sigma_{j-1} / sigma_j  (= beta_{j-1} sigma_{j-1})
  double acoef[kMaxKrylov];      // -alpha_j sigma_j (coefficient of U_j in U_{j+1})
  double psinorm;                // ||psi|| at the start of the step
  double psinorm0;               // batch: ||psi|| before the last combine (imaginary-time energy)
  double2 coef[kMaxKrylov];      // psi_new = sum_j coef_j U_j
  int kdim;                      // Krylov dimension kept
  int pad;
};

// Reduction workspace.
struct Reduction {
  double partial[kMaxPartials];
  unsigned int ticket;
  unsigned int pad[3];
  double normsq;                 // result of the last norm reduction
};

// Device-side status word bits.
enum : int { kStatusNonFinite = 1, kStatusTimeout = 2 };

struct Geometry {
  int N, L, stencil;
  int gauge = 0;                  // 0 length gauge (r E coupling), 1 velocity gauge (A p_z / c)
  int sms;                        // multiprocessors of the device (persistent grids)
  double dr;
  double c0, c1, c2;              // -1/2 d2/dr2 coefficients (c2 = 0 for 3 points)
};

// ---- launchers (tdse_kernels_fp64.cu) -------------------------------------
struct OperatorView {
  const double *diag, *rj, *kappa, *mask;
  const double *rinv = nullptr;   // 1 / r_j (velocity gauge)
  int mask_start;                 // first j index (0-based) with mask != 1; N if none
};

cudaError_t launch_apply_h(const Geometry &g, const OperatorView &op, double E,
                           const double2 *x, double2 *y, cudaStream_t s);
// imag: the stage of exp(-H dt) (imaginary time: -H instead of -i H, no mask).
cudaError_t launch_taylor_stage(const Geometry &g, const OperatorView &op, double E, double s,
                                const double2 *v_in, const double2 *psi, double2 *v_out,
                                bool final_stage, cudaStream_t st, bool imag = false);
cudaError_t launch_rk_stage(const Geometry &g, const OperatorView &op, double E, int stage,
                            double dt, const double2 *gin, const double2 *psi,
                            const double2 *acc_in, double2 *acc_out, double2 *g_next,
                            double2 *psi_out, cudaStream_t st, bool imag = false);
// One stage of an explicit Runge-Kutta method with up to kRkMaxStages stages
// (appendix "Runge-Kutta"): stage i computes k_i = -i H(E) g_i at every point
// (g_i = gin; g_0 is psi itself) and then, pointwise,
//   i < s-1: k_out = k_i,  g_out = psi + sum_{j<=i} coef[j] k_j  (coef = dt a_{i+1,j});
//   i = s-1: psi_out = mask * (psi + sum_j coef[j] k_j)           (coef = dt b_j, the
//            propagated weights), Delta = sum_j dcoef[j] k_j       (dcoef = dt (b_j - b^_j)),
//            *sigma += sqrt(sum |Delta|^2 / S) with S = (L+1) N (a grid reduction
//            in a fixed order; the last block adds it), and the status word
//            gets kStatusNonFinite when that sum is not finite (0 * Inf and
//            every sum with a NaN slope are NaN, so this also holds for the
//            methods whose b - bhat is zero).
// k[j] (j < i) are the stored slopes of the earlier stages; psi_out may be
// psi (each point is read before it is written by the same thread) but not gin.
// fsal (last stage only): the tableau is first-same-as-last (b_{s-1} = 0 and
// a_{s-1,j} = b_j), so psi + sum_j coef[j] k_j is gin itself and is not re-summed.
constexpr int kRkMaxStages = 7;
struct RkStageArgs {
  const double2 *k[kRkMaxStages];
  double2 *k_out, *g_out, *psi_out;
  double coef[kRkMaxStages], dcoef[kRkMaxStages];
  double *sigma;
  int *status;
  int stage, last, fsal;
};
cudaError_t launch_rk_general_stage(const Geometry &g, const OperatorView &op, double E,
                                    const double2 *gin, const double2 *psi, const RkStageArgs &a,
                                    Reduction *red, cudaStream_t st);
// ---- small grids: a whole run in one cluster launch (tdse_cluster.cu) --------
// Taylor, RK4 or Lanczos steps of an FP64 length-gauge grid small enough that
// the state and every work vector fit in the shared memory of one cluster of
// at most 16 CTAs (one per SM).  plan_small_grid picks the cluster (ctas CTAs,
// W radial columns each) or returns ok = false.  etab: the mid-step field per
// step (Taylor, Lanczos) or the fields at t_n, t_n + dt/2, t_n + dt (RK4).
// The Lanczos run leaves ||psi|| in ls (psinorm, sigma[0]) and red->normsq;
// a non-finite state sets kStatusNonFinite.
struct SmallPlan {
  bool ok = false;
  int ctas = 0, W = 0;
  size_t smem = 0;
};
SmallPlan plan_small_grid(const Geometry &g, int method, int order);
cudaError_t launch_small_grid(const SmallPlan &p, const Geometry &g, const OperatorView &op, int method,
                              int order, double dt, long nsteps, const double *etab, double2 *psi,
                              LanczosScalars *ls, Reduction *red, int *status, cudaStream_t st);
// ---- Sec. 4 dipole moments and flux (tdse_kernels_flux.cu) -------------------
// out[0..2] = <z>, d<z>/dt, d^2<z>/dt^2 of psi (E the field, ac = A/c in the
// velocity gauge else 0; the acceleration is NaN unless coulomb).  partials:
// 4 * dipole_blocks(g) doubles; ticket: zeroed, left zeroed.
int dipole_blocks(const Geometry &g);
cudaError_t launch_dipole_moments(const Geometry &g, const OperatorView &op, const double2 *psi,
                                  int ghost, double E, double ac, double Z, bool coulomb,
                                  double *partials, unsigned *ticket, double *out, cudaStream_t st);
// Flux through r = r_(ib+1) and its angular density at ntheta angles
// (ytab: Y_l0(theta_k), angle-major: ytab[k (L+1) + l]); state = {flux now, its integral, density now
// [ntheta], density integral [ntheta]}.  init: set "now" and zero the
// integrals; else integral += dt/2 (previous now + new now) first.
size_t flux_shared_bytes(const Geometry &g);
cudaError_t launch_flux(const Geometry &g, const OperatorView &op, const double2 *psi, int ghost,
                        int ib, double ac, const double *ytab, const double *cos_theta, int ntheta,
                        double dt, bool init, double *state, cudaStream_t st);
// Imaginary time: prev[0] = dr * red->normsq (the squared norm before a step);
// after the step (red->normsq of the new state): energy[0] =
// -ln(dr normsq / prev) / (2 dt) and psi /= sqrt(dr normsq).
cudaError_t launch_imag_begin(const Reduction *red, double dr, double *imag_dev, cudaStream_t st);
cudaError_t launch_imag_normalize(const Geometry &g, double2 *psi, const Reduction *red, double dt,
                                  double *imag_dev, cudaStream_t st);
cudaError_t launch_norm(const Geometry &g, const double2 *x, Reduction *red,
                        LanczosScalars *ls, int *status, cudaStream_t st);
cudaError_t launch_lanczos_a(const Geometry &g, const OperatorView &op, double E, int j,
                             const double2 *u, const double2 *uprev, double2 *z,
                             Reduction *red, LanczosScalars *ls, cudaStream_t st);
cudaError_t launch_lanczos_b(const Geometry &g, int j, const double2 *z, const double2 *u,
                             double2 *unext, Reduction *red, LanczosScalars *ls, cudaStream_t st);
// imag: c = exp(-T dt) e_1 (imaginary-time propagation) instead of exp(-i T dt) e_1.
cudaError_t launch_lanczos_expm(int m, double dt, LanczosScalars *ls, cudaStream_t st, bool imag = false);
// One block per listed instance: ids[0..count) index m, dt and ls (ids NULL:
// instances 0..count-1).
// Every Lanczos step of a call in one cooperative launch (tdse_persist.cu).
bool lanczos_persistent_fits(int stencil);
size_t lanczos_persistent_scratch_bytes();
cudaError_t launch_lanczos_persistent(const Geometry &g, const OperatorView &op, int m, double dt, long nsteps,
                                      const double *etab, double2 *psi, double2 *work, LanczosScalars *ls,
                                      Reduction *red, void *scratch, int *status, cudaStream_t st);
cudaError_t launch_lanczos_expm_batched(int count, const int *ids, const int *m, const double *dt, bool imag,
                                        LanczosScalars *ls, cudaStream_t st);
cudaError_t launch_lanczos_combine(const Geometry &g, const OperatorView &op, int m,
                                   double2 *psi, const double2 *work, size_t stride,
                                   Reduction *red, LanczosScalars *ls, int *status,
                                   cudaStream_t st);
// ---- mixed precision (tdse_kernels_mixed.cu) ------------------------------
struct MixedView {
  const float *diag;   // l(l+1)/(2 r^2) + V(r) (+ odd-ghost fold), without c0
  const float *rj, *kappa;
  const float *rinv;   // 1 / r_j (velocity gauge)
};

// hi/lo split of psi without the norm (the same split as every other kernel's)
cudaError_t launch_mx_split_plain(const Geometry &g, const double2 *psi, float2 *hi, float2 *lo, cudaStream_t st);
cudaError_t launch_mx_split(const Geometry &g, const double2 *psi, float2 *hi, float2 *lo,
                            Reduction *red, LanczosScalars *ls, int *status, cudaStream_t st);
cudaError_t launch_mx_apply_h(const Geometry &g, const MixedView &mv, double E, const double2 *x,
                              float2 *tmp_hi, float2 *tmp_lo, double2 *y, cudaStream_t st);
cudaError_t launch_mx_lanczos_a(const Geometry &g, const MixedView &mv, double E, int j,
                                const float2 *hi, const float2 *lo, const float2 *u,
                                const float2 *uprev, float2 *z, Reduction *red,
                                LanczosScalars *ls, cudaStream_t st);
cudaError_t launch_mx_lanczos_b(const Geometry &g, int j, const float2 *z, const float2 *u,
                                const float2 *hi, const float2 *lo, float2 *unext,
                                Reduction *red, LanczosScalars *ls, cudaStream_t st);
cudaError_t launch_mx_lanczos_combine(const Geometry &g, const OperatorView &op, double2 *psi,
                                      float2 *hi, float2 *lo, const float2 *u1, size_t stride,
                                      Reduction *red, LanczosScalars *ls, int *status,
                                      cudaStream_t st);
cudaError_t launch_mx_taylor_stage(const Geometry &g, const MixedView &mv, const OperatorView &op,
                                   double E, double s, const float2 *hi, const float2 *lo,
                                   const float2 *w_in, float2 *w_out, bool final_stage,
                                   double2 *psi, float2 *hi_out, float2 *lo_out, cudaStream_t st);
cudaError_t launch_mx_rk_stage(const Geometry &g, const MixedView &mv, const OperatorView &op,
                               double E, int stage, double dt, const float2 *hi, const float2 *lo,
                               const float2 *k_in, float2 *k_out, float2 *acc_hi, float2 *acc_lo,
                               double2 *psi, float2 *hi_out, float2 *lo_out, cudaStream_t st);

// partials: 5 * observables_blocks(g) * (L+1) doubles; ticket: a zeroed
// counter at a fixed address of the caller (left zeroed on return).
cudaError_t launch_observables(const Geometry &g, const OperatorView &op, const double2 *psi,
                               const double2 *ref0, double r_b, double *partials,
                               unsigned *ticket, double *out, cudaStream_t st);
int observables_blocks(const Geometry &g);

// ---- programmatic dependent launch -------------------------------------------
// The single-instance step is a chain of dependent kernels on one stream.  A
// kernel of the chain is launched with programmatic stream serialization
// (launch_pdl): the hardware may start its blocks while the kernel before it
// is still in its tail (the last block's grid reduction), which hides the
// launch and the block ramp.  Every such kernel calls pdl_wait() before its
// first access to device memory, which returns once the previous kernel has
// completed and its writes are visible (for a kernel launched without the
// attribute it returns at once); it calls pdl_trigger() when its main loop is
// done, which lets the next kernel launch.  The trigger always follows the
// wait, so at most two kernels of the chain are resident at a time.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<Args &&>(args)...);
}

}  // namespace tdse_dev
