// Green's function spectrum generation (FP64), see green.cu.
#pragma once
#include <cuda_runtime.h>

namespace flups {

constexpr int GL_N = 16;  // Gauss-Legendre nodes per quadrature panel

struct GreenSampleParams {
  int gext[3];        // Green index extents (x, y, z)
  int unb[3];         // 1: unbounded-like direction (sampled at r = g h), 0: spectral
  double h[3];        // grid spacing per direction
  double wscale[3];   // spectral wavenumber w = wscale (g + wshift)
  double wshift[3];
  int du;             // number of unbounded-like directions
  int kernel;         // 0 HEJ2m (order 2m, m = hej_m), 1 HEJ0
  int hej_m;          // m of HEJ2m (1 ... 5)
  double eps;         // regularisation length
  double hmax;        // HEJ0 cut-off spacing
  double gl_x[GL_N];  // Gauss-Legendre nodes and weights on [-1, 1]
  double gl_w[GL_N];
};

cudaError_t launch_green_sample(double* g, const GreenSampleParams& q, cudaStream_t st);
// Lattice Green's function samples G(n), n_d = 0..gext[d]-1 (every direction unbounded-like).
cudaError_t launch_lgf(double* g, const int* gext, const double* h, cudaStream_t st);
// n-point Gauss-Legendre nodes and weights on [-1, 1] (host).
void host_gauss_legendre(int n, double* x, double* w);
// out[(i / gx) gp + i % gx] = g[i] scale in the path precision (x rows of gx values at pitch gp)
cudaError_t launch_green_finalize(const double* g, void* out, int prec, long long n, int gx, int gp, double scale,
                                  cudaStream_t st);
cudaError_t launch_green_spectral(double* g, const int* gext, const double* const* tabs, int kernel, double eps2h,
                                  double scale, cudaStream_t st);
cudaError_t launch_special_eval(int which, const double* x, const double* y, double* out, int n, double eps,
                                const GreenSampleParams& q, cudaStream_t st);

}  // namespace flups
