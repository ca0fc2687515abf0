// Compile-time tile engine instantiations, double-float arithmetic, P >= 512.
#include <cuda_runtime.h>

#include "pass_kernels.cuh"

namespace flups {

cudaError_t launch_ct_df_large(int P, int kind, const PassParams& p, dim3 grid, int nthr, size_t smem,
                               cudaStream_t st) {
  switch (P) {
    case 512: return launch_kind<dfloat, 512, 8>(kind, p, grid, nthr, smem, st);
    case 1024: return launch_kind<dfloat, 1024, 4>(kind, p, grid, nthr, smem, st);
    case 2048: return launch_kind<dfloat, 2048, 2>(kind, p, grid, nthr, smem, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t set_limits_ct_df_large() {
  cudaError_t e = cudaSuccess;
  if (!e) e = set_limits_kind<dfloat, 512, 8>();
  if (!e) e = set_limits_kind<dfloat, 1024, 4>();
  if (!e) e = set_limits_kind<dfloat, 2048, 2>();
  return e;
}

}  // namespace flups
