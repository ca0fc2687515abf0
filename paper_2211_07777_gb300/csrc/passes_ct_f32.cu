// Compile-time tile engine instantiations, FP32 (P = 2^a, lanes per tile as ct_tile_width;
// P = 1024 in 4- and 8-lane tiles).
#include <cuda_runtime.h>

#include "pass_kernels.cuh"

namespace flups {

cudaError_t launch_ct_f32(int P, int kind, const PassParams& p, dim3 grid, int nthr, size_t smem, cudaStream_t st) {
  switch (P) {
    case 32: return launch_kind<float, 32, 64>(kind, p, grid, nthr, smem, st);
    case 64: return launch_kind<float, 64, 64>(kind, p, grid, nthr, smem, st);
    case 128: return launch_kind<float, 128, 32>(kind, p, grid, nthr, smem, st);
    case 256: return launch_kind<float, 256, 16>(kind, p, grid, nthr, smem, st);
    case 512: return launch_kind<float, 512, 16>(kind, p, grid, nthr, smem, st);
    case 1024: return p.W == 4 ? launch_kind<float, 1024, 4>(kind, p, grid, nthr, smem, st)
                               : launch_kind<float, 1024, 8>(kind, p, grid, nthr, smem, st);
    case 2048: return launch_kind<float, 2048, 4>(kind, p, grid, nthr, smem, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t set_limits_ct_f32() {
  cudaError_t e = cudaSuccess;
  if (!e) e = set_limits_kind<float, 32, 64>();
  if (!e) e = set_limits_kind<float, 64, 64>();
  if (!e) e = set_limits_kind<float, 128, 32>();
  if (!e) e = set_limits_kind<float, 256, 16>();
  if (!e) e = set_limits_kind<float, 512, 16>();
  if (!e) e = set_limits_kind<float, 1024, 8>();
  if (!e) e = set_limits_kind<float, 1024, 4>();
  if (!e) e = set_limits_kind<float, 2048, 4>();
  return e;
}

}  // namespace flups
