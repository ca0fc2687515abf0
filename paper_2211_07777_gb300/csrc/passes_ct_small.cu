// Compile-time tile engine, narrow tiles for small grids: FP32 P = 64 with 16 lanes.  A small grid
// has few pencils; narrow tiles spread them over more CTAs.  (Measured on GB300 against the
// runtime engine at 32^3-64^3: faster for FP32 at P = 64; slower for FP64 and double-float at
// P = 32, 64, whose short columns go to the runtime engine's warp-shuffle transforms or its
// radix-16 stages, and for FP32 at P = 32.)
#include <cuda_runtime.h>

#include "pass_kernels.cuh"

namespace flups {

int ct_small_width(int P, int prec) { return (prec == 0 && P == 64) ? 16 : 0; }

cudaError_t launch_ct_small(int prec, int P, int kind, const PassParams& p, dim3 grid, int nthr, size_t smem,
                            cudaStream_t st) {
  if (prec == 0 && P == 64) return launch_kind<float, 64, 16>(kind, p, grid, nthr, smem, st);
  return cudaErrorInvalidValue;
}

cudaError_t set_limits_ct_small() { return set_limits_kind<float, 64, 16>(); }

}  // namespace flups
