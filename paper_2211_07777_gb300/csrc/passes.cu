// Runtime-shaped pass kernels (any P = 2^a 3^b; FP32, FP64 and double-float) and the launch dispatch.
#include <cuda_runtime.h>

#include "pass_kernels.cuh"

namespace flups {

int ct_tile_width(int P, int prec, int axis, int kind) {
  // FP32 at P = 1024 (measured at 512^3): 4 lanes for the x passes (row mode) and for the
  // single-transform column passes (radix-32, 128 threads: more CTAs per SM to overlap their
  // memory phases); 8 lanes for the fused column pass and the other passes
  if (prec == 0 && P == 1024 && (axis == 0 || kind == K_FWD_C2C || kind == K_INV_C2C)) return 4;
  // lanes per tile: ~32-96 KB of shared memory, 16 elements per thread
  switch (P) {
    case 32: return prec == 0 ? 64 : 32;
    case 64: return prec == 0 ? 64 : 32;
    case 128: return prec == 0 ? 32 : 16;
    case 256: return prec == 0 ? 16 : 8;
    case 512: return prec == 0 ? 16 : 8;
    case 1024: return prec == 0 ? 8 : 4;
    case 2048: return prec == 0 ? 4 : 2;
  }
  return 0;
}

int ct_col_ept(int P, int prec, int kind) {
  // radix-32 stages (1024 = 32 x 32) for every FP32 column pass at P = 1024: the fused pass with
  // 8-lane tiles (256 threads), the single-transform passes with 4-lane tiles (128 threads)
  return (prec == 0 && P == 1024) ? 32 : 16;
}

cudaError_t set_pass_smem_limits() {
  cudaError_t e = set_limits_kind<float, 0, 0>();
  if (!e) e = set_limits_kind<double, 0, 0>();
  if (!e) e = set_limits_kind<dfloat, 0, 0>();
  if (!e) e = set_limits_ct_f32();
  if (!e) e = set_limits_ct_f64();
  if (!e) e = set_limits_ct_df();
  if (!e) e = set_limits_ct_small();
  return e;
}

cudaError_t launch_pass(int kind, int prec, const PassParams& p, dim3 grid, int nthr, size_t smem, cudaStream_t st) {
  if (p.ct && p.W == ct_small_width(p.P, prec)) return launch_ct_small(prec, p.P, kind, p, grid, nthr, smem, st);
  if (prec == 2) return p.ct ? launch_ct_df(p.P, kind, p, grid, nthr, smem, st)
                             : launch_kind<dfloat, 0, 0>(kind, p, grid, nthr, smem, st);
  if (p.ct) return prec == 0 ? launch_ct_f32(p.P, kind, p, grid, nthr, smem, st)
                             : launch_ct_f64(p.P, kind, p, grid, nthr, smem, st);
  return prec == 0 ? launch_kind<float, 0, 0>(kind, p, grid, nthr, smem, st)
                   : launch_kind<double, 0, 0>(kind, p, grid, nthr, smem, st);
}

}  // namespace flups
