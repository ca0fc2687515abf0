// Instruction-throughput microbenchmark: the measured FP32 and FP64 fused
// multiply-add rates of the device, the denominators of the arithmetic
// rooflines that the solve's FP64 and double-float passes are reported
// against.  No counterpart in the paper (measurement support).
//
// Every thread runs NCHAIN independent FMA chains (x = x * a + b) for ITER
// iterations, so that the FMA pipes see enough independent instructions to
// stay busy; the grid is a multiple of the SM count.  The chains' results are
// summed into one word per thread so that no FMA is dead code.
#include <cuda_runtime.h>

#include "flups_gpu.h"

namespace {

template <typename T, int NCHAIN>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, int iters, T a, T b) {
  T x[NCHAIN];
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < NCHAIN; ++c) x[c] = fma(x[c], a, b);
  }
  T s = (T)0;
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T, int NCHAIN>
int run_peak(int iters, double* tflops, double* ms_out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FLUPS_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FLUPS_ECUDA;
  const int threads = 256, blocks = sms * 8;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * threads * blocks) != cudaSuccess) return FLUPS_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // a and b keep x bounded (|a| < 1): no overflow or denormal slow path
  const T a = (T)0.999999, b = (T)1e-6;
  k_fma_peak<T, NCHAIN><<<blocks, threads>>>(out, iters / 8 + 1, a, b);  // warm-up
  cudaEventRecord(e0);
  k_fma_peak<T, NCHAIN><<<blocks, threads>>>(out, iters, a, b);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return FLUPS_ECUDA;
  const double fmas = (double)blocks * threads * (double)iters * 16.0 * NCHAIN;
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return FLUPS_OK;
}

}  // namespace

extern "C" int flups_measure_fma_peak(int prec, int iters, double* tflops, double* ms) {
  if (!tflops || iters < 1) return FLUPS_EINVAL;
  if (prec == FLUPS_F32) return run_peak<float, 8>(iters, tflops, ms);
  if (prec == FLUPS_F64) return run_peak<double, 8>(iters, tflops, ms);
  return FLUPS_EINVAL;
}
