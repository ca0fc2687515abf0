// Pass kernels of the solve: one launch per direction and sense.
//
// Every pass moves a tile of pencils through shared memory: gather from HBM
// (coalesced along x), build the periodic extension in shared memory (zero
// padding and symmetric images are never stored in HBM), complex FFT of the
// extension (fft_engine.cuh), then either store modes or -- in the fused last
// direction -- multiply by the Green's function spectrum and transform back.
//
// Real data are always transformed two pencils at a time: pencil a in the real
// part and pencil b in the imaginary part of one complex sequence, separated
// after the FFT through Hermitian symmetry (A_k = (Z_k + conj Z_{P-k})/2,
// B_k = (Z_k - conj Z_{P-k})/(2i)).  This serves the R2C DFT (Section 2.2,
// eq. sec2_dft_def) and the DCT/DST types I-IV of Table 1 alike: each r2r
// transform is read off the DFT of its even/odd extension, with the
// half-sample phase exp(-i pi k/P) for cell-centred data.
#include <cuda_runtime.h>

#include "pass_common.cuh"
#include "passes.cuh"

namespace flups {

// ---------------------------------------------------------------------------
// Forward pass on real data: R2C (periodic, doubled unbounded) or r2r
// coefficients (symmetric and semi-unbounded directions).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(MaxThreads<T>::value, 1) k_fwd_real(PassParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smraw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int W = p.W, LS = p.LS, P = p.P;
  const int q0 = blockIdx.x * 2 * W;
  const long long obase_i = (long long)blockIdx.y * p.ai.os + (long long)blockIdx.z * p.ai.cs;
  const long long obase_o = (long long)blockIdx.y * p.ao.os + (long long)blockIdx.z * p.ao.cs;
  const int ctype = comp_type(p, blockIdx.z);
  load_real_ext<T>(p, ctype, (const T*)p.in + obase_i, S, q0, tid, nthr);
  __syncthreads();
  const cpx<T>* tw = (const cpx<T>*)p.tw;
  S = fft_tile<T, false>(S, S + (size_t)P * LS, LS, P, W, p.lw, p.plan, tw, tid, nthr);

  const int t = base_type(ctype);
  const bool cplx_out = (t == T_PER || t == T_UNB);
  const bool quarter = is_quarter(t);
  const bool oddo = is_odd_origin(t);
  const bool cell = p.center == C_CELL;
  const int W2 = 2 * W, nm = p.n_modes;
  const int tot = nm * W2;
  const bool rowmode = p.axis == 0;
  for (int idx = tid; idx < tot; idx += nthr) {
    int c, k;
    if (rowmode) { k = idx % nm; c = idx / nm; } else { c = idx % W2; k = idx / W2; }
    const int q = q0 + c;
    if (q >= p.npen) continue;
    const int lane = c >> 1, part = c & 1;
    const int kk = quarter ? 2 * k + 1 : k;
    const int km = kk == 0 ? 0 : P - kk;
    const cpx<T> X = split<T>(S[kk * LS + lane], S[km * LS + lane], part);
    const long long off = (long long)q * p.ao.ls + (long long)k * p.ao.js;
    if (cplx_out) {
      ((cpx<T>*)p.out)[obase_o + off] = X;
    } else {
      cpx<T> F = X;
      if (cell) F = cmul<T>(X, __ldg(&tw[kk]));
      T v = oddo ? -F.y : F.x;
      if (quarter) v *= (T)0.5;
      ((T*)p.out)[obase_o + off] = v;
    }
  }
}

// Spectrum value X_kk of one pencil rebuilt from its stored modes (inverse of the above).
template <typename T>
__device__ __forceinline__ cpx<T> stored_mode(const PassParams& p, int type, const void* in, long long off_pencil,
                                              int kk, const cpx<T>* tw) {
  const int t = base_type(type);
  if (t == T_PER || t == T_UNB) {
    cpx<T> X = ((const cpx<T>*)in)[off_pencil + (long long)kk * p.ai.js];
    if (kk == 0 || 2 * kk == p.P) X.y = (T)0;  // DC and Nyquist of a real signal are real
    return X;
  }
  int m = kk;
  T div = (T)1;
  if (is_quarter(t)) {
    if ((kk & 1) == 0) return mk<T>((T)0, (T)0);
    m = (kk - 1) >> 1;
    div = (T)2;
  }
  const T c = ((const T*)in)[off_pencil + (long long)m * p.ai.js] * div;
  cpx<T> F = is_odd_origin(t) ? mk<T>((T)0, -c) : mk<T>(c, (T)0);
  if (p.center == C_CELL) F = cmulc<T>(F, __ldg(&tw[kk]));
  return F;
}

template <typename T>
__global__ void __launch_bounds__(MaxThreads<T>::value, 1) k_inv_real(PassParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smraw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int W = p.W, LS = p.LS, P = p.P;
  const int q0 = blockIdx.x * 2 * W;
  const long long obase_i = (long long)blockIdx.y * p.ai.os + (long long)blockIdx.z * p.ai.cs;
  const long long obase_o = (long long)blockIdx.y * p.ao.os + (long long)blockIdx.z * p.ao.cs;
  const cpx<T>* tw = (const cpx<T>*)p.tw;
  const int ctype = comp_type(p, blockIdx.z);
  const int half = P / 2;
  const int tot = (half + 1) * W;
  const bool rowmode = p.axis == 0;
  for (int idx = tid; idx < tot; idx += nthr) {
    int lane, k;
    if (rowmode) { k = idx % (half + 1); lane = idx / (half + 1); } else { lane = idx % W; k = idx / W; }
    const int qa = q0 + 2 * lane, qb = qa + 1;
    cpx<T> Xa = mk<T>((T)0, (T)0), Xb = Xa;
    if (qa < p.npen) Xa = stored_mode<T>(p, ctype, p.in, obase_i + (long long)qa * p.ai.ls, k, tw);
    if (qb < p.npen) Xb = stored_mode<T>(p, ctype, p.in, obase_i + (long long)qb * p.ai.ls, k, tw);
    S[k * LS + lane] = mk<T>(Xa.x - Xb.y, Xa.y + Xb.x);
    if (k != 0 && 2 * k != P) S[(P - k) * LS + lane] = mk<T>(Xa.x + Xb.y, Xb.x - Xa.y);
  }
  __syncthreads();
  S = fft_tile<T, true>(S, S + (size_t)P * LS, LS, P, W, p.lw, p.plan, tw, tid, nthr);
  store_real_data<T>(p, ctype, (T*)p.out + obase_o, S, q0, tid, nthr);
}

// ---------------------------------------------------------------------------
// Complex passes (second and third complex directions).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(MaxThreads<T>::value, 1) k_fwd_c2c(PassParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smraw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int W = p.W, LS = p.LS, P = p.P;
  const int q0 = blockIdx.x * W;
  const long long obase_i = (long long)blockIdx.y * p.ai.os + (long long)blockIdx.z * p.ai.cs;
  const long long obase_o = (long long)blockIdx.y * p.ao.os + (long long)blockIdx.z * p.ao.cs;
  load_cplx<T>(p, (const cpx<T>*)p.in + obase_i, S, q0, tid, nthr);
  __syncthreads();
  S = fft_tile<T, false>(S, S + (size_t)P * LS, LS, P, W, p.lw, p.plan, (const cpx<T>*)p.tw, tid, nthr);
  cpx<T>* out = (cpx<T>*)p.out + obase_o;
  const int tot = P * W;
  const bool rowmode = p.axis == 0;
  for (int idx = tid; idx < tot; idx += nthr) {
    int lane, k;
    if (rowmode) { k = idx % P; lane = idx / P; } else { lane = idx % W; k = idx / W; }
    const int q = q0 + lane;
    if (q >= p.npen) continue;
    out[(long long)q * p.ao.ls + (long long)k * p.ao.js] = S[k * LS + lane];
  }
}

template <typename T>
__global__ void __launch_bounds__(MaxThreads<T>::value, 1) k_inv_c2c(PassParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smraw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int W = p.W, LS = p.LS, P = p.P;
  const int q0 = blockIdx.x * W;
  const long long obase_i = (long long)blockIdx.y * p.ai.os + (long long)blockIdx.z * p.ai.cs;
  const long long obase_o = (long long)blockIdx.y * p.ao.os + (long long)blockIdx.z * p.ao.cs;
  const cpx<T>* in = (const cpx<T>*)p.in + obase_i;
  const int tot = P * W;
  const bool rowmode = p.axis == 0;
  for (int idx = tid; idx < tot; idx += nthr) {
    int lane, k;
    if (rowmode) { k = idx % P; lane = idx / P; } else { lane = idx % W; k = idx / W; }
    const int q = q0 + lane;
    cpx<T> v = mk<T>((T)0, (T)0);
    if (q < p.npen) v = in[(long long)q * p.ai.ls + (long long)k * p.ai.js];
    S[k * LS + lane] = v;
  }
  __syncthreads();
  S = fft_tile<T, true>(S, S + (size_t)P * LS, LS, P, W, p.lw, p.plan, (const cpx<T>*)p.tw, tid, nthr);
  store_cplx_data<T>(p, (cpx<T>*)p.out + obase_o, S, q0, tid, nthr);
}

// ---------------------------------------------------------------------------
// Fused last direction: forward FFT, times G^, inverse FFT (u^ = G^ f^, eq. poisson).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T green_closed(int kernel, T k2, T eps2h, T scale) {
  if (!(k2 > (T)0)) return (T)0;
  if (kernel == 0 || kernel == 100) return -scale / k2;
  const int m = kernel / 2;
  const T s = k2 * eps2h;
  T acc = (T)1, term = (T)1;
  for (int j = 1; j < m; ++j) {
    term = term * s / (T)j;
    acc += term;
  }
  return -scale * exp(-s) * acc / k2;
}

// Green index of a pencil along the two non-axis directions: stored offset
// (without the axis term) or the closed-form partial |k|^2.
template <typename T>
__device__ __forceinline__ void pencil_green_base(const PassParams& p, int q, int o, long long* goff, T* k2p) {
  const FusedGreen& g = p.g;
  if (q >= p.npen) {  // ragged tile: no pencil, no Green access
    *goff = 0;
    *k2p = (T)0;
    return;
  }
  int c[3];
  if (p.axis == 0) { c[1] = q % g.dims1; c[2] = q / g.dims1; c[0] = 0; }
  else if (p.axis == 1) { c[0] = q; c[2] = o; c[1] = 0; }
  else { c[0] = q; c[1] = o; c[2] = 0; }
  long long off = 0;
  T k2 = (T)0;
  const long long st[3] = {1, (long long)g.gext[0], (long long)g.gext[0] * g.gext[1]};
  for (int d = 0; d < 3; ++d) {
    if (d == p.axis) continue;
    int gi = c[d];
    if (g.fold[d]) gi = min(gi, g.fold[d] - gi);
    off += gi * st[d];
    if (!g.stored) k2 += ((const T*)g.tab[d])[gi];
  }
  *goff = off;
  *k2p = k2;
}

template <typename T>
__device__ __forceinline__ T green_at(const PassParams& p, long long goff, T k2p, int g3) {
  const FusedGreen& g = p.g;
  if (g.stored) {
    const long long st3 = p.axis == 0 ? 1 : (p.axis == 1 ? (long long)g.gext[0] : (long long)g.gext[0] * g.gext[1]);
    return __ldg(&((const T*)g.stored)[goff + g3 * st3]);
  }
  const T k2 = k2p + ((const T*)g.tab[p.axis])[g3];
  return green_closed<T>(g.kernel, k2, (T)g.eps2_half, (T)g.scale);
}

template <typename T>
__global__ void __launch_bounds__(MaxThreads<T>::value, 1) k_fused_c2c(PassParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smraw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int W = p.W, LS = p.LS, P = p.P;
  cpx<T>* S2 = S + (size_t)P * LS;
  long long* goff = reinterpret_cast<long long*>(smraw + 2 * (size_t)P * LS * sizeof(cpx<T>));
  T* k2p = reinterpret_cast<T*>(goff + W);
  const int q0 = blockIdx.x * W;
  const long long obase = (long long)blockIdx.y * p.ai.os + (long long)blockIdx.z * p.ai.cs;
  for (int lane = tid; lane < W; lane += nthr) pencil_green_base<T>(p, q0 + lane, blockIdx.y, &goff[lane], &k2p[lane]);
  load_cplx<T>(p, (const cpx<T>*)p.in + obase, S, q0, tid, nthr);
  __syncthreads();
  const cpx<T>* tw = (const cpx<T>*)p.tw;
  cpx<T>* X = fft_tile<T, false>(S, S2, LS, P, W, p.lw, p.plan, tw, tid, nthr);
  const int tot = P * W;
  for (int idx = tid; idx < tot; idx += nthr) {
    const int lane = idx % W, k = idx / W;
    const int g3 = min(k, P - k);
    const T G = green_at<T>(p, goff[lane], k2p[lane], g3);
    X[k * LS + lane] = cscale<T>(X[k * LS + lane], G);
  }
  __syncthreads();
  X = fft_tile<T, true>(X, X == S ? S2 : S, LS, P, W, p.lw, p.plan, tw, tid, nthr);
  store_cplx_data<T>(p, (cpx<T>*)p.out + obase, X, q0, tid, nthr);
}

template <typename T>
__global__ void __launch_bounds__(MaxThreads<T>::value, 1) k_fused_real(PassParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smraw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int W = p.W, LS = p.LS, P = p.P;
  cpx<T>* S2 = S + (size_t)P * LS;
  long long* goff = reinterpret_cast<long long*>(smraw + 2 * (size_t)P * LS * sizeof(cpx<T>));
  T* k2p = reinterpret_cast<T*>(goff + 2 * W);
  const int q0 = blockIdx.x * 2 * W;
  const long long obase = (long long)blockIdx.y * p.ai.os + (long long)blockIdx.z * p.ai.cs;
  for (int c = tid; c < 2 * W; c += nthr) pencil_green_base<T>(p, q0 + c, blockIdx.y, &goff[c], &k2p[c]);
  const int ctype = comp_type(p, blockIdx.z);
  load_real_ext<T>(p, ctype, (const T*)p.in + obase, S, q0, tid, nthr);
  __syncthreads();
  const cpx<T>* tw = (const cpx<T>*)p.tw;
  cpx<T>* X = fft_tile<T, false>(S, S2, LS, P, W, p.lw, p.plan, tw, tid, nthr);
  const bool quarter = is_quarter(base_type(ctype));
  const int half = P / 2;
  const int tot = (half + 1) * W;
  for (int idx = tid; idx < tot; idx += nthr) {
    const int lane = idx % W, k = idx / W;
    const int km = k == 0 ? 0 : P - k;
    const cpx<T> zk = X[k * LS + lane], zm = X[km * LS + lane];
    cpx<T> A = split<T>(zk, zm, 0), B = split<T>(zk, zm, 1);
    if (quarter && (k & 1) == 0) {
      A = mk<T>((T)0, (T)0);
      B = A;
    } else {
      const int g3 = quarter ? (k - 1) >> 1 : k;
      const T Ga = green_at<T>(p, goff[2 * lane], k2p[2 * lane], g3);
      const T Gb = green_at<T>(p, goff[2 * lane + 1], k2p[2 * lane + 1], g3);
      A = cscale<T>(A, Ga);
      B = cscale<T>(B, Gb);
    }
    X[k * LS + lane] = mk<T>(A.x - B.y, A.y + B.x);
    if (k != 0 && 2 * k != P) X[km * LS + lane] = mk<T>(A.x + B.y, B.x - A.y);
  }
  __syncthreads();
  X = fft_tile<T, true>(X, X == S ? S2 : S, LS, P, W, p.lw, p.plan, tw, tid, nthr);
  store_real_data<T>(p, ctype, (T*)p.out + obase, X, q0, tid, nthr);
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
template <typename T>
static cudaError_t set_limits_t() {
  const int lim = 227 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_fwd_real<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_inv_real<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_fwd_c2c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_inv_c2c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_fused_real<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  return cudaFuncSetAttribute(k_fused_c2c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

cudaError_t set_pass_smem_limits() {
  cudaError_t e = set_limits_t<float>();
  if (e) return e;
  return set_limits_t<double>();
}

template <typename T>
static void launch_t(int kind, const PassParams& p, dim3 grid, int nthr, size_t smem, cudaStream_t st) {
  switch (kind) {
    case K_FWD_REAL: k_fwd_real<T><<<grid, nthr, smem, st>>>(p); break;
    case K_INV_REAL: k_inv_real<T><<<grid, nthr, smem, st>>>(p); break;
    case K_FWD_C2C: k_fwd_c2c<T><<<grid, nthr, smem, st>>>(p); break;
    case K_INV_C2C: k_inv_c2c<T><<<grid, nthr, smem, st>>>(p); break;
    case K_FUSED_REAL: k_fused_real<T><<<grid, nthr, smem, st>>>(p); break;
    case K_FUSED_C2C: k_fused_c2c<T><<<grid, nthr, smem, st>>>(p); break;
  }
}

cudaError_t launch_pass(int kind, int prec, const PassParams& p, dim3 grid, int nthr, size_t smem, cudaStream_t st) {
  if (prec == 0) launch_t<float>(kind, p, grid, nthr, smem, st);
  else launch_t<double>(kind, p, grid, nthr, smem, st);
  return cudaGetLastError();
}

}  // namespace flups
