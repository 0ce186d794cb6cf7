// Launchers of the small exponential exp(-i T dt) e_1 (see tdse_small_expm.cuh).
#include <cuda_runtime.h>

#include <cmath>

#include "tdse_small_expm.cuh"

namespace tdse_dev {

// The single-instance step's kernel chain launches this one with programmatic
// serialization (launch_pdl): it waits for the Lanczos iterations, then lets
// the combine's blocks launch at once (they wait for it in turn).
__global__ void __launch_bounds__(kEx) lanczos_expm_kernel(int m, double dt, LanczosScalars *ls, int imag) {
  pdl_wait();
  pdl_trigger();
  expm_body(m, dt, ls, imag != 0);
}

// One block per listed instance of a batch (ids[b], or b when ids is null).
__global__ void __launch_bounds__(kEx)
    lanczos_expm_batched_kernel(const int *__restrict__ ids, const int *__restrict__ m,
                                const double *__restrict__ dt, LanczosScalars *ls, int imag) {
  const int i = ids ? ids[blockIdx.x] : (int)blockIdx.x;
  expm_body(m[i], dt[i], ls + i, imag != 0);
}

cudaError_t launch_lanczos_expm(int m, double dt, LanczosScalars *ls, cudaStream_t st, bool imag) {
  if (!st) {   // the legacy default stream: an ordinary launch
    lanczos_expm_kernel<<<1, kEx, 0, st>>>(m, dt, ls, imag ? 1 : 0);
    return cudaGetLastError();
  }
  const cudaError_t e = launch_pdl(lanczos_expm_kernel, 1, kEx, 0, st, m, dt, ls, imag ? 1 : 0);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_lanczos_expm_batched(int count, const int *ids, const int *m, const double *dt, bool imag,
                                        LanczosScalars *ls, cudaStream_t st) {
  if (count < 1) return cudaSuccess;
  lanczos_expm_batched_kernel<<<count, kEx, 0, st>>>(ids, m, dt, ls, imag ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace tdse_dev

// ---- the small exponential on its own (C ABI, include/tdse.h) ---------------
extern "C" int tdse_lanczos_expm(int m, const double *alpha, const double *beta, double dt, int imag,
                                 double *c_out, int *kdim) {
  using namespace tdse_dev;
  if (m < 1 || m > kMaxKrylov || !alpha || (m > 1 && !beta) || !c_out || !(dt > 0.0) || !std::isfinite(dt))
    return TDSE_ERR_ARG;
  LanczosScalars h{};
  for (int j = 0; j < m; ++j) h.alpha[j] = alpha[j];
  for (int j = 0; j + 1 < m; ++j) h.beta[j] = beta[j];
  // psi_new = sum_j c_j q_j with ||psi|| = 1 and sigma_j = 1: coef_j = c_j
  h.psinorm = 1.0;
  for (int j = 0; j <= kMaxKrylov; ++j) h.sigma[j] = 1.0;
  LanczosScalars *d = nullptr;
  if (cudaMalloc(&d, sizeof(LanczosScalars)) != cudaSuccess) {
    cudaGetLastError();
    return TDSE_ERR_OOM;
  }
  cudaError_t e = cudaMemcpy(d, &h, sizeof(h), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_lanczos_expm(m, dt, d, nullptr, imag != 0);
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return TDSE_ERR_CUDA;
  for (int j = 0; j < m; ++j) {
    c_out[2 * j] = (j < h.kdim) ? h.coef[j].x : 0.0;
    c_out[2 * j + 1] = (j < h.kdim) ? h.coef[j].y : 0.0;
  }
  if (kdim) *kdim = h.kdim;
  return TDSE_OK;
}
