// Launchers of the small exponential exp(-i T dt) e_1 (see tdse_small_expm.cuh).
#include <cuda_runtime.h>

#include "tdse_small_expm.cuh"

namespace tdse_dev {

__global__ void __launch_bounds__(kEx) lanczos_expm_kernel(int m, double dt, LanczosScalars *ls, int imag) {
  expm_body(m, dt, ls, imag != 0);
}

// One block per listed instance of a batch (ids[b], or b when ids is null).
__global__ void __launch_bounds__(kEx)
    lanczos_expm_batched_kernel(const int *__restrict__ ids, const int *__restrict__ m,
                                const double *__restrict__ dt, LanczosScalars *ls) {
  const int i = ids ? ids[blockIdx.x] : (int)blockIdx.x;
  expm_body(m[i], dt[i], ls + i);
}

cudaError_t launch_lanczos_expm(int m, double dt, LanczosScalars *ls, cudaStream_t st, bool imag) {
  lanczos_expm_kernel<<<1, kEx, 0, st>>>(m, dt, ls, imag ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_lanczos_expm_batched(int count, const int *ids, const int *m, const double *dt,
                                        LanczosScalars *ls, cudaStream_t st) {
  if (count < 1) return cudaSuccess;
  lanczos_expm_batched_kernel<<<count, kEx, 0, st>>>(ids, m, dt, ls);
  return cudaGetLastError();
}

}  // namespace tdse_dev
