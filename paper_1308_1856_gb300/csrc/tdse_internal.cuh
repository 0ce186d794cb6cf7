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

#include <string>
#include <vector>

#include "../../include/tdse.h"

namespace tdse_dev {

constexpr int kMaxKrylov = TDSE_MAX_KRYLOV;
constexpr int kBlockJ = 128;            // threads per block of the stencil kernels
constexpr int kStencilBlocksPerSM = 8;  // persistent stencil grid: 8 x 4 warps per SM
constexpr int kElemBlocksPerSM = 4;     // persistent elementwise grid: 4 x 8 warps per SM
constexpr int kMaxPartials = 16384;     // block partial slots of one grid reduction

// Scalars of one Lanczos step, resident in device memory.
struct LanczosScalars {
  double alpha[kMaxKrylov];      // alpha_j = <q_j, H q_j>
  double beta[kMaxKrylov];       // beta_j = ||w_j|| (beta[j] links q_j and q_{j+1})
  double sigma[kMaxKrylov + 1];  // sigma_j = 1 / ||U_j||  (U_0 = psi, U_j unnormalised)
  double psinorm;                // ||psi|| at the start of the step
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
enum : int { kStatusNonFinite = 1 };

struct Geometry {
  int N, L, stencil;
  int sms;                        // multiprocessors of the device (persistent grids)
  double dr;
  double c0, c1, c2;              // -1/2 d2/dr2 coefficients (c2 = 0 for 3 points)
};

// ---- launchers (tdse_kernels_fp64.cu) -------------------------------------
struct OperatorView {
  const double *diag, *rj, *kappa, *mask;
  int mask_start;                 // first j index (0-based) with mask != 1; N if none
};

cudaError_t launch_apply_h(const Geometry &g, const OperatorView &op, double E,
                           const double2 *x, double2 *y, cudaStream_t s);
cudaError_t launch_taylor_stage(const Geometry &g, const OperatorView &op, double E, double s,
                                const double2 *v_in, const double2 *psi, double2 *v_out,
                                bool final_stage, cudaStream_t st);
cudaError_t launch_rk_stage(const Geometry &g, const OperatorView &op, double E, int stage,
                            double dt, const double2 *gin, const double2 *psi,
                            const double2 *acc_in, double2 *acc_out, double2 *g_next,
                            double2 *psi_out, cudaStream_t st);
cudaError_t launch_norm(const Geometry &g, const double2 *x, Reduction *red,
                        LanczosScalars *ls, int *status, cudaStream_t st);
cudaError_t launch_lanczos_a(const Geometry &g, const OperatorView &op, double E, int j,
                             const double2 *u, const double2 *uprev, double2 *z,
                             Reduction *red, LanczosScalars *ls, cudaStream_t st);
cudaError_t launch_lanczos_b(const Geometry &g, int j, const double2 *z, const double2 *u,
                             double2 *unext, Reduction *red, LanczosScalars *ls, cudaStream_t st);
cudaError_t launch_lanczos_expm(int m, double dt, LanczosScalars *ls, cudaStream_t st);
cudaError_t launch_lanczos_combine(const Geometry &g, const OperatorView &op, int m,
                                   double2 *psi, const double2 *work, size_t stride,
                                   Reduction *red, LanczosScalars *ls, int *status,
                                   cudaStream_t st);
cudaError_t launch_observables(const Geometry &g, const OperatorView &op, const double2 *psi,
                               const double2 *ref0, double r_b, double *partials, int nq,
                               double *out, cudaStream_t st);
int observables_blocks(const Geometry &g);

}  // namespace tdse_dev
