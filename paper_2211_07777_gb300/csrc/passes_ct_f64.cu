// Compile-time tile engine instantiations, FP64 (P = 2^a, lanes per tile as ct_tile_width).
#include <cuda_runtime.h>

#include "pass_kernels.cuh"

namespace flups {

cudaError_t launch_ct_f64(int P, int kind, const PassParams& p, dim3 grid, int nthr, size_t smem, cudaStream_t st) {
  switch (P) {
    case 32: return launch_kind<double, 32, 32>(kind, p, grid, nthr, smem, st);
    case 64: return launch_kind<double, 64, 32>(kind, p, grid, nthr, smem, st);
    case 128: return launch_kind<double, 128, 16>(kind, p, grid, nthr, smem, st);
    case 256: return launch_kind<double, 256, 8>(kind, p, grid, nthr, smem, st);
    case 512: return launch_kind<double, 512, 8>(kind, p, grid, nthr, smem, st);
    case 1024: return launch_kind<double, 1024, 4>(kind, p, grid, nthr, smem, st);
    case 2048: return launch_kind<double, 2048, 2>(kind, p, grid, nthr, smem, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t set_limits_ct_f64() {
  cudaError_t e = cudaSuccess;
  if (!e) e = set_limits_kind<double, 32, 32>();
  if (!e) e = set_limits_kind<double, 64, 32>();
  if (!e) e = set_limits_kind<double, 128, 16>();
  if (!e) e = set_limits_kind<double, 256, 8>();
  if (!e) e = set_limits_kind<double, 512, 8>();
  if (!e) e = set_limits_kind<double, 1024, 4>();
  if (!e) e = set_limits_kind<double, 2048, 2>();
  return e;
}

}  // namespace flups
