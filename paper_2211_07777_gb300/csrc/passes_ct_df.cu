// Compile-time tile engine instantiations, double-float arithmetic (the FP64-class
// emulated path; same tile widths as FP64, same bytes per element).  P <= 256 here,
// P >= 512 in passes_ct_df_large.cu (two translation units compile in parallel).
#include <cuda_runtime.h>

#include "pass_kernels.cuh"

namespace flups {

cudaError_t launch_ct_df(int P, int kind, const PassParams& p, dim3 grid, int nthr, size_t smem, cudaStream_t st) {
  switch (P) {
    case 32: return launch_kind<dfloat, 32, 32>(kind, p, grid, nthr, smem, st);
    case 64: return launch_kind<dfloat, 64, 32>(kind, p, grid, nthr, smem, st);
    case 128: return launch_kind<dfloat, 128, 16>(kind, p, grid, nthr, smem, st);
    case 256: return launch_kind<dfloat, 256, 8>(kind, p, grid, nthr, smem, st);
  }
  return launch_ct_df_large(P, kind, p, grid, nthr, smem, st);
}

cudaError_t set_limits_ct_df() {
  cudaError_t e = cudaSuccess;
  if (!e) e = set_limits_kind<dfloat, 32, 32>();
  if (!e) e = set_limits_kind<dfloat, 64, 32>();
  if (!e) e = set_limits_kind<dfloat, 128, 16>();
  if (!e) e = set_limits_kind<dfloat, 256, 8>();
  if (!e) e = set_limits_ct_df_large();
  return e;
}

}  // namespace flups
