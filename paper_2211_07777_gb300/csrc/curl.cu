// Fused last direction of the Biot-Savart solve, lap(u) = curl(f) (Section
// "Application: the Biot-Savart solver", eq. biotsavart): forward transform of
// the three components of a pencil, u^ = G^ (i w x f^) in spectral space, and
// the inverse transform of each velocity component with its own conditions.
//
// Derivatives (same section): along a periodic or unbounded direction the
// stored modes are complex and d/dx -> i sigma(w).  Along an even/odd
// direction the stored coefficients are real: a cosine-type coefficient c
// (even at the origin) becomes -sigma c of the sine-type output, a sine-type
// coefficient becomes +sigma c of the cosine-type output -- the sign rule of
// the paper, which also holds for the quarter-wave and semi-unbounded types
// (common mode index).  sigma is the spectral symbol w or the finite-difference
// symbols of order 2, 4, 6, tabulated per extension mode in FP64.  Along the
// fused direction the derivative acts on the extension's DFT directly.
#include <cuda_runtime.h>

#include <type_traits>

#include "pass_common.cuh"

namespace flups {

template <typename T> struct CurlMaxThreads { static constexpr int value = 512; };
template <> struct CurlMaxThreads<double> { static constexpr int value = 256; };
template <> struct CurlMaxThreads<dfloat> { static constexpr int value = 256; };

// Per-pencil data: Green access and the derivative factors of the two non-axis
// directions for each source component: fac[d][c] (complex).
template <typename T>
struct PencilCurl {
  long long goff;
  T k2p;
  cpx<T> fac[3][3];
};

template <typename T>
__device__ __forceinline__ void pencil_curl_setup(const PassParams& p, int q, int o, PencilCurl<T>* pc) {
  const FusedGreen& g = p.g;
  for (int d = 0; d < 3; ++d)
    for (int c = 0; c < 3; ++c) pc->fac[d][c] = mk<T>((T)0, (T)0);
  if (q >= p.npen) {
    pc->goff = 0;
    pc->k2p = (T)0;
    return;
  }
  int crd[3];
  if (p.axis == 0) { crd[1] = q % g.dims1; crd[2] = q / g.dims1; crd[0] = 0; }
  else if (p.axis == 1) { crd[0] = q; crd[2] = o; crd[1] = 0; }
  else { crd[0] = q; crd[1] = o; crd[2] = 0; }
  long long off = 0;
  T k2 = (T)0;
  const long long st[3] = {1, (long long)g.gpitch, (long long)g.gpitch * g.gext[1]};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (d == p.axis) continue;
    const int m = crd[d];
    int gi = m;
    if (g.fold[d]) gi = min(gi, g.fold[d] - gi);
    off += gi * st[d];
    if (!g.stored) k2 += ((const T*)g.tab[d])[gi];
    const int kk = (g.role[d] == 0 && g.quarter[d]) ? 2 * m + 1 : m;
    const T s = ((const T*)g.dsym[d])[kk];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (g.role[d] == 0) pc->fac[d][c] = mk<T>(((g.srcodd[d] >> c) & 1) ? s : -s, (T)0);
      else pc->fac[d][c] = mk<T>((T)0, s);
    }
  }
  pc->goff = off;
  pc->k2p = k2;
}

template <typename T>
__device__ __forceinline__ T curl_green(const PassParams& p, const PencilCurl<T>& pc, int g3) {
  const FusedGreen& g = p.g;
  if constexpr (!std::is_same<T, dfloat>::value) {
    if (!g.stored) {
      const T k2 = pc.k2p + ((const T*)g.tab[p.axis])[g3];
      if (!(k2 > (T)0)) return (T)0;
      if (g.kernel == 0 || g.kernel == 100) return -(T)g.scale / k2;
      const int m = g.kernel / 2;
      const T s = k2 * (T)g.eps2_half;
      T acc = (T)1, term = (T)1;
      for (int j = 1; j < m; ++j) {
        term = term * s / (T)j;
        acc += term;
      }
      return -(T)g.scale * exp(-s) * acc / k2;
    }
  }
  // stored spectrum (always, on the double-float path)
  const long long st3 = p.axis == 0 ? 1 : (p.axis == 1 ? (long long)g.gpitch : (long long)g.gpitch * g.gext[1]);
  return ldg_r<T>(&((const T*)g.stored)[pc.goff + g3 * st3]);
}

// u_c = G (D_a f_b - D_b f_a), (a, b) = (c + 1, c + 2): F holds f^ of the pencil at one mode.
template <typename T>
__device__ __forceinline__ void curl_mode(const PassParams& p, const PencilCurl<T>& pc, cpx<T> d3, T G,
                                          const cpx<T>* F, cpx<T>* U) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int a = (c + 1) % 3, b = (c + 2) % 3;
    const cpx<T> Dab = (a == p.axis) ? d3 : pc.fac[a][b];
    const cpx<T> Dba = (b == p.axis) ? d3 : pc.fac[b][a];
    const cpx<T> t = csub<T>(cmul<T>(Dab, F[b]), cmul<T>(Dba, F[a]));
    U[c] = cscale<T>(t, G);
  }
}

template <typename T>
__device__ __forceinline__ int ext_green_index(int k, int P, bool quarter) {
  const int f = min(k, P - k);
  return quarter ? max(f - 1, 0) >> 1 : f;
}

// Real data on all three components (the earlier directions were r2r): two
// pencils per complex FFT, as in the scalar fused pass.
template <typename T>
__global__ void __launch_bounds__(CurlMaxThreads<T>::value, 1) k_curl_real(PassParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int W = p.W, LS = p.LS, P = p.P;
  const size_t buf = (size_t)P * LS;
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smraw);   // 3 components x 2 buffers
  PencilCurl<T>* pcs = reinterpret_cast<PencilCurl<T>*>(smraw + 6 * buf * sizeof(cpx<T>));
  const int q0 = blockIdx.x * 2 * W;
  const long long obase = (long long)blockIdx.y * p.ai.os;
  for (int c = tid; c < 2 * W; c += nthr) pencil_curl_setup<T>(p, q0 + c, blockIdx.y, &pcs[c]);
  for (int c = 0; c < 3; ++c)
    load_real_ext<T>(p, comp_type(p, c), (const T*)p.in + obase + c * p.ai.cs, S + 2 * c * buf, q0, tid, nthr);
  __syncthreads();
  const cpx<T>* tw = (const cpx<T>*)p.tw;
  cpx<T>* X[3];
  for (int c = 0; c < 3; ++c) X[c] = fft_tile<T, false>(S + 2 * c * buf, S + (2 * c + 1) * buf, LS, P, W, p.lw, p.plan, tw, tid, nthr);
  const bool quarter = is_quarter(base_type(comp_type(p, 0)));
  const T* sym3 = (const T*)p.g.dsym[p.axis];
  const int half = P / 2;
  const int tot = (half + 1) * W;
  for (int idx = tid; idx < tot; idx += nthr) {
    const int lane = idx % W, k = idx / W;
    const int km = k == 0 ? 0 : P - k;
    cpx<T> A[3], B[3], UA[3], UB[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cpx<T> zk = X[c][k * LS + lane], zm = X[c][km * LS + lane];
      A[c] = split<T>(zk, zm, 0);
      B[c] = split<T>(zk, zm, 1);
    }
    if (quarter && (k & 1) == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) UA[c] = UB[c] = mk<T>((T)0, (T)0);
    } else {
      const int g3 = ext_green_index<T>(k, P, quarter);
      const cpx<T> d3 = mk<T>((T)0, sym3[k]);
      const PencilCurl<T>& pa = pcs[2 * lane];
      const PencilCurl<T>& pb = pcs[2 * lane + 1];
      curl_mode<T>(p, pa, d3, curl_green<T>(p, pa, g3), A, UA);
      curl_mode<T>(p, pb, d3, curl_green<T>(p, pb, g3), B, UB);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      X[c][k * LS + lane] = mk<T>(UA[c].x - UB[c].y, UA[c].y + UB[c].x);
      if (k != 0 && 2 * k != P) X[c][km * LS + lane] = mk<T>(UA[c].x + UB[c].y, UB[c].x - UA[c].y);
    }
  }
  __syncthreads();
  for (int c = 0; c < 3; ++c) {
    cpx<T>* other = (X[c] == S + 2 * c * buf) ? S + (2 * c + 1) * buf : S + 2 * c * buf;
    cpx<T>* R = fft_tile<T, true>(X[c], other, LS, P, W, p.lw, p.plan, tw, tid, nthr);
    store_real_data<T>(p, (p.g.utypes >> (4 * c)) & 15, (T*)p.out + obase + c * p.ao.cs, R, q0, tid, nthr);
  }
}

// Complex data (an earlier direction was periodic or unbounded): one pencil per lane.
template <typename T>
__global__ void __launch_bounds__(CurlMaxThreads<T>::value, 1) k_curl_c2c(PassParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int W = p.W, LS = p.LS, P = p.P;
  const size_t buf = (size_t)P * LS;
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smraw);
  PencilCurl<T>* pcs = reinterpret_cast<PencilCurl<T>*>(smraw + 6 * buf * sizeof(cpx<T>));
  const int q0 = blockIdx.x * W;
  const long long obase = (long long)blockIdx.y * p.ai.os;
  for (int c = tid; c < W; c += nthr) pencil_curl_setup<T>(p, q0 + c, blockIdx.y, &pcs[c]);
  for (int c = 0; c < 3; ++c) load_cplx<T>(p, (const cpx<T>*)p.in + obase + c * p.ai.cs, S + 2 * c * buf, q0, tid, nthr);
  __syncthreads();
  const cpx<T>* tw = (const cpx<T>*)p.tw;
  cpx<T>* X[3];
  for (int c = 0; c < 3; ++c) X[c] = fft_tile<T, false>(S + 2 * c * buf, S + (2 * c + 1) * buf, LS, P, W, p.lw, p.plan, tw, tid, nthr);
  const T* sym3 = (const T*)p.g.dsym[p.axis];
  const int tot = P * W;
  for (int idx = tid; idx < tot; idx += nthr) {
    const int lane = idx % W, k = idx / W;
    cpx<T> F[3], U[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) F[c] = X[c][k * LS + lane];
    const PencilCurl<T>& pc = pcs[lane];
    curl_mode<T>(p, pc, mk<T>((T)0, sym3[k]), curl_green<T>(p, pc, min(k, P - k)), F, U);
#pragma unroll
    for (int c = 0; c < 3; ++c) X[c][k * LS + lane] = U[c];
  }
  __syncthreads();
  for (int c = 0; c < 3; ++c) {
    cpx<T>* other = (X[c] == S + 2 * c * buf) ? S + (2 * c + 1) * buf : S + 2 * c * buf;
    cpx<T>* R = fft_tile<T, true>(X[c], other, LS, P, W, p.lw, p.plan, tw, tid, nthr);
    store_cplx_data<T>(p, (cpx<T>*)p.out + obase + c * p.ao.cs, R, q0, tid, nthr);
  }
}

template <typename T>
static cudaError_t set_curl_limits_t() {
  const int lim = 227 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_curl_real<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e) return e;
  return cudaFuncSetAttribute(k_curl_c2c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

cudaError_t set_curl_smem_limits() {
  cudaError_t e = set_curl_limits_t<float>();
  if (!e) e = set_curl_limits_t<double>();
  if (!e) e = set_curl_limits_t<dfloat>();
  return e;
}

cudaError_t launch_curl(int kind, int prec, const PassParams& p, dim3 grid, int nthr, size_t smem, cudaStream_t st) {
  if (prec == 0) {
    if (kind == K_CURL_REAL) k_curl_real<float><<<grid, nthr, smem, st>>>(p);
    else k_curl_c2c<float><<<grid, nthr, smem, st>>>(p);
  } else if (prec == 2) {
    if (kind == K_CURL_REAL) k_curl_real<dfloat><<<grid, nthr, smem, st>>>(p);
    else k_curl_c2c<dfloat><<<grid, nthr, smem, st>>>(p);
  } else {
    if (kind == K_CURL_REAL) k_curl_real<double><<<grid, nthr, smem, st>>>(p);
    else k_curl_c2c<double><<<grid, nthr, smem, st>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace flups
