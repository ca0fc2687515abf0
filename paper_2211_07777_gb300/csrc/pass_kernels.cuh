// Pass kernels of the solve, as templates over the arithmetic type T and the
// tile shape: PC = 0 takes the FFT length and tile width from the parameters
// (runtime engine, any P = 2^a 3^b, ping-pong buffers); PC = P > 0 compiles
// the whole tile for P = 2^a and WC lanes (compile-time engine, in place).
//
// Every pass moves a tile of pencils through shared memory: gather from HBM
// (coalesced along x), build the periodic extension in shared memory (zero
// padding and symmetric images are never stored in HBM), complex FFT of the
// extension, then either store modes or -- in the fused last direction --
// multiply by the Green's function spectrum and transform back.
//
// Real data are always transformed two pencils at a time: pencil a in the real
// part and pencil b in the imaginary part of one complex sequence, separated
// after the FFT through Hermitian symmetry (A_k = (Z_k + conj Z_{P-k})/2,
// B_k = (Z_k - conj Z_{P-k})/(2i)).  This serves the R2C DFT (Section 2.2,
// eq. sec2_dft_def) and the DCT/DST types I-IV of Table 1 alike: each r2r
// transform is read off the DFT of its even/odd extension, with the
// half-sample phase exp(-i pi k/P) for cell-centred data.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "pass_common.cuh"
#include "passes.cuh"

namespace flups {

// Launch bounds: the runtime engine runs at most 512 (FP32) / 256 (FP64)
// threads; the compile-time engine exactly P W / 16, and is built for 1024 (FP32) or 512 threads
// per SM (a CTA narrower than a warp holds a whole warp's registers).
template <typename T, int PC, int WC> struct KBounds {
  static constexpr int threads = PC ? PC * WC / 16 : (sizeof(T) == 4 ? 512 : 256);
  static constexpr int wthreads = threads < 32 ? 32 : threads;
  static constexpr int minb = PC ? ((sizeof(T) == 4 ? 1024 : 512) / wthreads > 0 ? (sizeof(T) == 4 ? 1024 : 512) / wthreads : 1) : 1;
};

// Column kernels: EPT elements per thread and stage (16, or 32 with radix-32 stages), so
// P W / EPT threads; with EPT = 32 a thread may use up to 128 registers (2 CTAs of 256 threads per SM).
template <typename T, int PC, int WC, int EPT> struct ColBounds {
  static constexpr int threads = PC * WC / EPT;
  static constexpr int minb = EPT == 32 ? (512 / threads > 0 ? 512 / threads : 1) : KBounds<T, PC, WC>::minb;
};

template <typename T, int PC, int WC>
struct Tile {
  static constexpr bool CT = PC > 0;
  __device__ __forceinline__ static int P(const PassParams& p) { return CT ? PC : p.P; }
  __device__ __forceinline__ static int W(const PassParams& p) { return CT ? WC : p.W; }
  __device__ __forceinline__ static int LS(const PassParams& p) { return CT ? WC + 1 : p.LS; }
  __device__ __forceinline__ static int lw(const PassParams& p) { return CT ? clog2(WC) : p.lw; }
};

// FFT of the tile held in S (S2 = second buffer of the runtime engine); returns the buffer holding the result.
template <typename T, int PC, int WC, bool INV, bool ZIN = false, bool ZOUT = false>
__device__ __forceinline__ cpx<T>* run_fft(const PassParams& p, cpx<T>* S, cpx<T>* S2, const cpx<T>* tw, int tid,
                                           int nthr) {
  if constexpr (PC > 0) {
    fft_tile_ct<T, PC, WC, INV, ZIN, ZOUT>(S, tw, tid);
    return S;
  } else {
    if (warp_fft_len(p.P)) {
      fft_tile_warp<T, INV>(S, p.LS, p.P, p.W, tw, tid, nthr);
      return S;
    }
    return fft_tile<T, INV>(S, S2, p.LS, p.P, p.W, p.lw, p.plan, tw, tid, nthr);
  }
}

template <typename T, int PC>
__device__ __forceinline__ cpx<T>* second_buffer(const PassParams& p, cpx<T>* S) {
  return PC > 0 ? S : S + (size_t)p.P * p.LS;
}

// Spectrum value X_kk of one pencil rebuilt from its stored modes (inverse of the forward store).
template <typename T>
__device__ __forceinline__ cpx<T> stored_mode(const PassParams& p, int type, const void* in, long long off_pencil,
                                              int kk, int P, const cpx<T>* tw) {
  const int t = base_type(type);
  if (t == T_PER || t == T_UNB) {
    cpx<T> X = ((const cpx<T>*)in)[off_pencil + (long long)kk * p.ai.js];
    if (kk == 0 || 2 * kk == P) X.y = (T)0;  // DC and Nyquist of a real signal are real
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
  if (p.center == C_CELL) F = cmulc<T>(F, ldg_c<T>(&tw[kk]));
  return F;
}

// ---------------------------------------------------------------------------
// Forward pass on real data: R2C (periodic, doubled unbounded) or r2r
// coefficients (symmetric and semi-unbounded directions).
// ---------------------------------------------------------------------------
template <typename T, int PC, int WC, bool HZ>
__global__ void __launch_bounds__(KBounds<T, PC, WC>::threads, KBounds<T, PC, WC>::minb) k_fwd_real(PassParams p) {
  pass_entry(p);
  extern __shared__ __align__(16) unsigned char smraw[];
  using TL = Tile<T, PC, WC>;
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smraw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int W = TL::W(p), LS = TL::LS(p), P = TL::P(p);
  const int q0 = blockIdx.x * 2 * W;
  const long long obase_i = (long long)blockIdx.y * p.ai.os + (long long)blockIdx.z * p.ai.cs;
  const long long obase_o = (long long)blockIdx.y * p.ao.os + (long long)blockIdx.z * p.ao.cs;
  const int ctype = comp_type(p, blockIdx.z);
  load_real_ext<T, WC>(p, ctype, (const T*)p.in + obase_i, S, q0, tid, nthr, HZ);
  __syncthreads();
  const cpx<T>* tw = (const cpx<T>*)p.tw;

  const int t = base_type(ctype);
  const bool cplx_out = (t == T_PER || t == T_UNB);
  const bool quarter = is_quarter(t);
  const bool oddo = is_odd_origin(t);
  const bool cell = p.center == C_CELL;
  const int W2 = 2 * W, nm = p.n_modes;
  const bool rowmode = p.axis == 0;
  auto store_mode = [&](int q, int k, int kk, const cpx<T>& X) {
    const long long off = (long long)q * p.ao.ls + (long long)k * p.ao.js;
    if (cplx_out) {
      ((cpx<T>*)p.out)[obase_o + off] = X;
    } else {
      cpx<T> F = X;
      if (cell) F = cmul<T>(X, ldg_c<T>(&tw[kk]));
      T v = oddo ? -F.y : F.x;
      if (quarter) v = v * T(0.5);
      st_real<T>((T*)p.out, obase_o + off, v, p.out_f64);
    }
  };
  if constexpr (PC == 0) {
    if (warp_fft_len(P)) {
      // short columns: the lane holding mode kk takes the mirrored mode P - kk from the lane that
      // holds it, separates the two packed pencils and stores both coefficients from registers
      const int lgP = 31 - __clz(P);
      fft_cols_warp<T, false>(S, LS, P, W, tw, tid, nthr, [&](int c, int kk, const cpx<T>& zk, bool ok) {
        const int km = kk == 0 ? 0 : P - kk;
        const int src = ((tid & 31) & ~(P - 1)) | (int)(__brev((unsigned)km) >> (32 - lgP));
        const cpx<T> zm = shfl_idx_c<T>(zk, src);
        if (!ok || (quarter && !(kk & 1))) return;
        const int k = quarter ? (kk - 1) >> 1 : kk;
        if (k >= nm) return;
        for (int part = 0; part < 2; ++part) {
          const int q = q0 + 2 * c + part;
          if (q < p.npen) store_mode(q, k, kk, split<T>(zk, zm, part));
        }
      });
      return;
    }
  }
  S = run_fft<T, PC, WC, false, HZ, false>(p, S, second_buffer<T, PC>(p, S), tw, tid, nthr);
  if (PC > 0 && rowmode) {
    // compile-time tile in row mode: a thread reads Z_k and Z_{P-k} of a lane once and stores the
    // mode of both of its pencils; modes k < P/2 as W rows of P/2 (8 per thread, k fastest), then
    // k = P/2 (every type has at most P/2 + 1 modes) on threads tid < W
    const int tot = W * (P / 2) + nthr;
    for (int idx = tid; idx < tot; idx += nthr) {
      int lane, k;
      if (idx < W * (P / 2)) { lane = idx / (P / 2); k = idx % (P / 2); }
      else { lane = idx - W * (P / 2); k = P / 2; if (lane >= W) continue; }
      if (k >= nm) continue;
      const int qa = q0 + 2 * lane;
      if (qa >= p.npen) continue;
      const int kk = quarter ? 2 * k + 1 : k;
      const int km = kk == 0 ? 0 : P - kk;
      const cpx<T> zk = S[tix<T, WC>(kk, lane, LS)], zm = S[tix<T, WC>(km, lane, LS)];
      store_mode(qa, k, kk, split<T>(zk, zm, 0));
      if (qa + 1 < p.npen) store_mode(qa + 1, k, kk, split<T>(zk, zm, 1));
    }
    return;
  }
  const int tot = rowmode ? (W2 << p.ndlog) : nm * W2;
  for (int idx = tid; idx < tot; idx += nthr) {
    int c, k;
    if (rowmode) { k = idx & ((1 << p.ndlog) - 1); c = idx >> p.ndlog; if (k >= nm) continue; }
    else { c = idx & (W2 - 1); k = idx >> (TL::lw(p) + 1); }
    const int q = q0 + c;
    if (q >= p.npen) continue;
    const int lane = c >> 1, part = c & 1;
    const int kk = quarter ? 2 * k + 1 : k;
    const int km = kk == 0 ? 0 : P - kk;
    store_mode(q, k, kk, split<T>(S[tix<T, WC>(kk, lane, LS)], S[tix<T, WC>(km, lane, LS)], part));
  }
}

template <typename T, int PC, int WC, bool HZ>
__global__ void __launch_bounds__(KBounds<T, PC, WC>::threads, KBounds<T, PC, WC>::minb) k_inv_real(PassParams p) {
  pass_entry(p);
  extern __shared__ __align__(16) unsigned char smraw[];
  using TL = Tile<T, PC, WC>;
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smraw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int W = TL::W(p), LS = TL::LS(p), P = TL::P(p);
  const int q0 = blockIdx.x * 2 * W;
  const long long obase_i = (long long)blockIdx.y * p.ai.os + (long long)blockIdx.z * p.ai.cs;
  const long long obase_o = (long long)blockIdx.y * p.ao.os + (long long)blockIdx.z * p.ao.cs;
  const cpx<T>* tw = (const cpx<T>*)p.tw;
  const int ctype = comp_type(p, blockIdx.z);
  const int half = P / 2;
  const bool rowmode = p.axis == 0;
  // (not on the double-float path, whose registers do not hold 18 modes per thread)
  constexpr bool BATCH = PC > 0 && !std::is_same<T, dfloat>::value;
  if (BATCH && rowmode) {
    // compile-time tile in row mode: the W x P/2 modes k < P/2 are exactly 8 per thread
    // (NT = P W / 16), loaded in batches of IB per thread (both pencils' modes of a lane);
    // lane = idx / (P/2) keeps k fastest (coalesced); the Nyquist modes k = P/2 go to threads
    // tid < W with the last batch
    constexpr int HP = PC / 2, NB8 = 8, IB = 4;
    // with p.rows_bulk the CTA's rows q0 .. q0 + 2W - 1 (complex modes, rows p.ai.ls apart) are first
    // copied into shared memory by one bulk copy, and the modes are read from there
    const cpx<T>* rows = nullptr;
    if (p.rows_bulk) {
      unsigned char* sb = smraw + p.rows_off;
      unsigned long long* bar = reinterpret_cast<unsigned long long*>(sb) - 16;
      const int nrows = min(2 * W, p.npen - q0);
      if (tid == 0) mbar_init(bar, 1);
      __syncthreads();
      if (tid == 0) {
        const unsigned bytes = (unsigned)((size_t)nrows * p.ai.ls * sizeof(cpx<T>));
        mbar_expect_tx(bar, bytes);
        bulk_load(sb, (const cpx<T>*)p.in + obase_i + (long long)q0 * p.ai.ls, bytes, bar);
      }
      const bool ok = mbar_wait_bounded(bar, p.errflag, 2, p.dbg_wait & 2);
      if (__syncthreads_or(!ok)) return;  // the tile's input did not arrive in time: no stores
      rows = reinterpret_cast<const cpx<T>*>(sb);
    }
    auto mode = [&](int q, int k) -> cpx<T> {
      if (!rows) return stored_mode<T>(p, ctype, p.in, obase_i + (long long)q * p.ai.ls, k, P, tw);
      cpx<T> X = rows[(long long)(q - q0) * p.ai.ls + k];
      if (k == 0 || 2 * k == P) X.y = (T)0;  // DC and Nyquist of a real signal are real
      return X;
    };
#pragma unroll
    for (int u0 = 0; u0 < NB8; u0 += IB) {
      constexpr int NI = IB + 1;
      cpx<T> Xa[NI], Xb[NI];
      const bool last = u0 + IB == NB8;
#pragma unroll
      for (int e = 0; e < NI; ++e) {
        const int u = u0 + e;
        const bool nyq = e == IB;
        const int idx = tid + u * nthr;
        const int lane = nyq ? tid : idx / HP, k = nyq ? HP : idx % HP;
        const int qa = q0 + 2 * lane, qb = qa + 1;
        Xa[e] = mk<T>((T)0, (T)0);
        Xb[e] = Xa[e];
        if (nyq && !(last && tid < W)) continue;
        if (qa < p.npen) Xa[e] = mode(qa, k);
        if (qb < p.npen) Xb[e] = mode(qb, k);
      }
#pragma unroll
      for (int e = 0; e < NI; ++e) {
        const int u = u0 + e;
        const bool nyq = e == IB;
        if (nyq && !(last && tid < W)) continue;
        const int idx = tid + u * nthr;
        const int lane = nyq ? tid : idx / HP, k = nyq ? HP : idx % HP;
        S[tix<T, WC>(k, lane, LS)] = mk<T>(Xa[e].x - Xb[e].y, Xa[e].y + Xb[e].x);
        if (k != 0 && 2 * k != P) S[tix<T, WC>(P - k, lane, LS)] = mk<T>(Xa[e].x + Xb[e].y, Xb[e].x - Xa[e].y);
      }
    }
  }
  // row mode: k fastest over a power-of-two stride (1 << p.hlog) >= half + 1
  const int tot = (BATCH && rowmode) ? 0 : (rowmode ? (W << p.hlog) : (half + 1) * W);
  constexpr int LOADB = 4;
  for (int base = tid; base < tot; base += LOADB * nthr) {
    cpx<T> Xa[LOADB], Xb[LOADB];
    int ll[LOADB], kk[LOADB];
#pragma unroll
    for (int u = 0; u < LOADB; ++u) {
      const int idx = base + u * nthr;
      int lane = 0, k = -1;
      if (idx < tot) {
        if (rowmode) { k = idx & ((1 << p.hlog) - 1); lane = idx >> p.hlog; if (k > half) k = -1; }
        else { lane = idx & (W - 1); k = idx >> TL::lw(p); }
      }
      ll[u] = lane;
      kk[u] = k;
      const int qa = q0 + 2 * lane, qb = qa + 1;
      Xa[u] = mk<T>((T)0, (T)0);
      Xb[u] = Xa[u];
      if (k >= 0 && qa < p.npen) Xa[u] = stored_mode<T>(p, ctype, p.in, obase_i + (long long)qa * p.ai.ls, k, P, tw);
      if (k >= 0 && qb < p.npen) Xb[u] = stored_mode<T>(p, ctype, p.in, obase_i + (long long)qb * p.ai.ls, k, P, tw);
    }
#pragma unroll
    for (int u = 0; u < LOADB; ++u) {
      const int k = kk[u];
      if (k < 0) continue;
      const int lane = ll[u];
      S[tix<T, WC>(k, lane, LS)] = mk<T>(Xa[u].x - Xb[u].y, Xa[u].y + Xb[u].x);
      if (k != 0 && 2 * k != P) S[tix<T, WC>(P - k, lane, LS)] = mk<T>(Xa[u].x + Xb[u].y, Xb[u].x - Xa[u].y);
    }
  }
  __syncthreads();
  if constexpr (PC == 0) {
    if (warp_fft_len(P) && p.center == C_CELL) {
      // short columns of cell-centred data (data index = extension position, or its reversal): the
      // lane holding position pos stores that value of both packed pencils from registers
      const bool rev = is_reversed(ctype);
      const int nd = p.n_data;
      T* out = (T*)p.out + obase_o;
      fft_cols_warp<T, true>(S, LS, P, W, tw, tid, nthr, [&](int c, int pos, const cpx<T>& z, bool ok) {
        if (!ok || pos >= nd) return;
        const long long off = (long long)(rev ? nd - 1 - pos : pos) * p.ao.js;
        const int qa = q0 + 2 * c;
        if (qa < p.npen) st_real<T>(out, (long long)qa * p.ao.ls + off, z.x, p.out_f64);
        if (qa + 1 < p.npen) st_real<T>(out, (long long)(qa + 1) * p.ao.ls + off, z.y, p.out_f64);
      });
      return;
    }
  }
  S = run_fft<T, PC, WC, true, false, HZ>(p, S, second_buffer<T, PC>(p, S), tw, tid, nthr);
  store_real_data<T, WC>(p, ctype, (T*)p.out + obase_o, S, q0, tid, nthr);
}

// ---------------------------------------------------------------------------
// Complex passes (second and third complex directions).
// ---------------------------------------------------------------------------

// Store of an inverse complex pass from the lane holding extension position i of pencil q (the
// element-wise form of store_cplx_data): data index i < n_data, and node-centred periodic
// phi_N := phi_0.
template <typename T>
__device__ __forceinline__ void store_cplx_at(const PassParams& p, cpx<T>* out, int q, int i, const cpx<T>& v) {
  if (q >= p.npen) return;
  const long long row = (long long)q * p.ao.ls;
  if (i < p.n_data) out[row + (long long)i * p.ao.js] = v;
  if (i == 0 && p.type == T_PER && p.center == C_NODE && p.N < p.n_data) out[row + (long long)p.N * p.ao.js] = v;
}
template <typename T, int PC, int WC, bool HZ>
__global__ void __launch_bounds__(KBounds<T, PC, WC>::threads, KBounds<T, PC, WC>::minb) k_fwd_c2c(PassParams p) {
  pass_entry(p);
  extern __shared__ __align__(16) unsigned char smraw[];
  using TL = Tile<T, PC, WC>;
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smraw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int W = TL::W(p), LS = TL::LS(p), P = TL::P(p);
  const int q0 = blockIdx.x * W;
  const long long obase_i = (long long)blockIdx.y * p.ai.os + (long long)blockIdx.z * p.ai.cs;
  const long long obase_o = (long long)blockIdx.y * p.ao.os + (long long)blockIdx.z * p.ao.cs;
  load_cplx<T, WC>(p, (const cpx<T>*)p.in + obase_i, S, q0, tid, nthr, HZ);
  __syncthreads();
  cpx<T>* out = (cpx<T>*)p.out + obase_o;
  if constexpr (PC == 0) {
    if (warp_fft_len(P)) {  // short columns: modes stored from the lanes' registers
      fft_cols_warp<T, false>(S, LS, P, W, (const cpx<T>*)p.tw, tid, nthr,
                              [&](int c, int k, const cpx<T>& v, bool ok) {
                                const int q = q0 + c;
                                if (ok && q < p.npen) out[(long long)q * p.ao.ls + (long long)k * p.ao.js] = v;
                              });
      return;
    }
  }
  S = run_fft<T, PC, WC, false, HZ, false>(p, S, second_buffer<T, PC>(p, S), (const cpx<T>*)p.tw, tid, nthr);
  const bool rowmode = p.axis == 0;
  const int tot = P * W;
  for (int idx = tid; idx < tot; idx += nthr) {
    int lane, k;
    if (rowmode) { k = idx % P; lane = idx / P; } else { lane = idx & (W - 1); k = idx >> TL::lw(p); }
    const int q = q0 + lane;
    if (q >= p.npen) continue;
    out[(long long)q * p.ao.ls + (long long)k * p.ao.js] = S[tix<T, WC>(k, lane, LS)];
  }
}

template <typename T, int PC, int WC, bool HZ>
__global__ void __launch_bounds__(KBounds<T, PC, WC>::threads, KBounds<T, PC, WC>::minb) k_inv_c2c(PassParams p) {
  pass_entry(p);
  extern __shared__ __align__(16) unsigned char smraw[];
  using TL = Tile<T, PC, WC>;
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smraw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int W = TL::W(p), LS = TL::LS(p), P = TL::P(p);
  const int q0 = blockIdx.x * W;
  const long long obase_i = (long long)blockIdx.y * p.ai.os + (long long)blockIdx.z * p.ai.cs;
  const long long obase_o = (long long)blockIdx.y * p.ao.os + (long long)blockIdx.z * p.ao.cs;
  const cpx<T>* in = (const cpx<T>*)p.in + obase_i;
  const bool rowmode = p.axis == 0;
  const int tot = P * W;
  for (int idx = tid; idx < tot; idx += nthr) {
    int lane, k;
    if (rowmode) { k = idx % P; lane = idx / P; } else { lane = idx & (W - 1); k = idx >> TL::lw(p); }
    const int q = q0 + lane;
    cpx<T> v = mk<T>((T)0, (T)0);
    if (q < p.npen) v = in[(long long)q * p.ai.ls + (long long)k * p.ai.js];
    S[tix<T, WC>(k, lane, LS)] = v;
  }
  __syncthreads();
  if constexpr (PC == 0) {
    if (warp_fft_len(P)) {  // short columns: data stored from the lanes' registers
      cpx<T>* out = (cpx<T>*)p.out + obase_o;
      fft_cols_warp<T, true>(S, LS, P, W, (const cpx<T>*)p.tw, tid, nthr, [&](int c, int k, const cpx<T>& v, bool ok) {
        if (ok) store_cplx_at<T>(p, out, q0 + c, k, v);
      });
      return;
    }
  }
  S = run_fft<T, PC, WC, true, false, HZ>(p, S, second_buffer<T, PC>(p, S), (const cpx<T>*)p.tw, tid, nthr);
  store_cplx_data<T, WC>(p, (cpx<T>*)p.out + obase_o, S, q0, tid, nthr);
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
  const long long st[3] = {1, (long long)g.gpitch, (long long)g.gpitch * g.gext[1]};
#pragma unroll
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
  if constexpr (!std::is_same<T, dfloat>::value) {
    if (!g.stored) {
      const T k2 = k2p + ((const T*)g.tab[p.axis])[g3];
      return green_closed<T>(g.kernel, k2, (T)g.eps2_half, (T)g.scale);
    }
  }
  // stored spectrum (always, on the double-float path)
  const long long st3 = p.axis == 0 ? 1 : (p.axis == 1 ? (long long)g.gpitch : (long long)g.gpitch * g.gext[1]);
  return ldg_r<T>(&((const T*)g.stored)[goff + g3 * st3]);
}

template <typename T, int PC>
__device__ __forceinline__ size_t tile_bytes(const PassParams& p) {
  return (PC > 0 ? 1 : 2) * (size_t)p.P * p.LS * sizeof(cpx<T>);
}

template <typename T, int PC, int WC, bool HZ>
__global__ void __launch_bounds__(KBounds<T, PC, WC>::threads, KBounds<T, PC, WC>::minb) k_fused_c2c(PassParams p) {
  pass_entry(p);
  extern __shared__ __align__(16) unsigned char smraw[];
  using TL = Tile<T, PC, WC>;
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smraw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int W = TL::W(p), LS = TL::LS(p), P = TL::P(p);
  cpx<T>* S2 = second_buffer<T, PC>(p, S);
  long long* goff = reinterpret_cast<long long*>(smraw + tile_bytes<T, PC>(p));
  T* k2p = reinterpret_cast<T*>(goff + W);
  const int q0 = blockIdx.x * W;
  const long long obase = (long long)blockIdx.y * p.ai.os + (long long)blockIdx.z * p.ai.cs;
  for (int lane = tid; lane < W; lane += nthr) pencil_green_base<T>(p, q0 + lane, blockIdx.y, &goff[lane], &k2p[lane]);
  load_cplx<T, WC>(p, (const cpx<T>*)p.in + obase, S, q0, tid, nthr, HZ);
  __syncthreads();
  const cpx<T>* tw = (const cpx<T>*)p.tw;
  if constexpr (PC == 0) {
    if (warp_fft_len(P)) {  // short columns: both transforms, the product and the store from registers
      cpx<T>* out = (cpx<T>*)p.out + obase;
      conv_cols_warp<T>(S, LS, P, W, tw, tid, nthr,
                        [&](int c, int k) { return green_at<T>(p, goff[c], k2p[c], min(k, P - k)); },
                        [&](int c, int i, const cpx<T>& v) { store_cplx_at<T>(p, out, q0 + c, i, v); });
      return;
    }
  }
  cpx<T>* X = run_fft<T, PC, WC, false, HZ, false>(p, S, S2, tw, tid, nthr);
  const int tot = P * W;
  for (int idx = tid; idx < tot; idx += nthr) {
    const int lane = idx & (W - 1), k = idx >> TL::lw(p);
    const int g3 = min(k, P - k);
    const T G = green_at<T>(p, goff[lane], k2p[lane], g3);
    X[tix<T, WC>(k, lane, LS)] = cscale<T>(X[tix<T, WC>(k, lane, LS)], G);
  }
  __syncthreads();
  X = run_fft<T, PC, WC, true, false, HZ>(p, X, X == S ? S2 : S, tw, tid, nthr);
  store_cplx_data<T, WC>(p, (cpx<T>*)p.out + obase, X, q0, tid, nthr);
}

template <typename T, int PC, int WC, bool HZ>
__global__ void __launch_bounds__(KBounds<T, PC, WC>::threads, KBounds<T, PC, WC>::minb) k_fused_real(PassParams p) {
  pass_entry(p);
  extern __shared__ __align__(16) unsigned char smraw[];
  using TL = Tile<T, PC, WC>;
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smraw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int W = TL::W(p), LS = TL::LS(p), P = TL::P(p);
  cpx<T>* S2 = second_buffer<T, PC>(p, S);
  long long* goff = reinterpret_cast<long long*>(smraw + tile_bytes<T, PC>(p));
  T* k2p = reinterpret_cast<T*>(goff + 2 * W);
  const int q0 = blockIdx.x * 2 * W;
  const long long obase = (long long)blockIdx.y * p.ai.os + (long long)blockIdx.z * p.ai.cs;
  for (int c = tid; c < 2 * W; c += nthr) pencil_green_base<T>(p, q0 + c, blockIdx.y, &goff[c], &k2p[c]);
  const int ctype = comp_type(p, blockIdx.z);
  load_real_ext<T, WC>(p, ctype, (const T*)p.in + obase, S, q0, tid, nthr, HZ);
  __syncthreads();
  const cpx<T>* tw = (const cpx<T>*)p.tw;
  cpx<T>* X = run_fft<T, PC, WC, false, HZ, false>(p, S, S2, tw, tid, nthr);
  const bool quarter = is_quarter(base_type(ctype));
  const int half = P / 2;
  const int tot = (half + 1) * W;
  for (int idx = tid; idx < tot; idx += nthr) {
    const int lane = idx & (W - 1), k = idx >> TL::lw(p);
    const int km = k == 0 ? 0 : P - k;
    const cpx<T> zk = X[tix<T, WC>(k, lane, LS)], zm = X[tix<T, WC>(km, lane, LS)];
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
    X[tix<T, WC>(k, lane, LS)] = mk<T>(A.x - B.y, A.y + B.x);
    if (k != 0 && 2 * k != P) X[tix<T, WC>(km, lane, LS)] = mk<T>(A.x + B.y, B.x - A.y);
  }
  __syncthreads();
  X = run_fft<T, PC, WC, true, false, HZ>(p, X, X == S ? S2 : S, tw, tid, nthr);
  store_real_data<T, WC>(p, ctype, (T*)p.out + obase, X, q0, tid, nthr);
}

// ---------------------------------------------------------------------------
// Column-mode compile-time kernels (complex passes along y or z): the first
// stage reads its butterfly inputs straight from HBM into registers (loads
// coalesced across the W lanes = consecutive x), the last stage stores
// straight from registers to HBM, and the fused pass keeps the last forward
// stage's outputs in registers, multiplies them by G^ and runs the first
// inverse stage on them -- the inverse plan takes the radices in reverse
// order so that its first butterflies read exactly those elements.  Shared
// memory carries only the exchanges between stages.
// ---------------------------------------------------------------------------
enum XsMode : int { XS_SMEM = 0, XS_GLOBAL = 1, XS_REGS = 2, XS_NAT = 3 };  // XS_NAT: dense rows (TMA tile)

template <typename T>
struct ColIO {
  const cpx<T>* in;
  cpx<T>* out;
  long long ils, ijs, ols, ojs;
  int q0, npen;
  int n_in, n_out;  // rows read (the rest is zero padding) and rows written (truncation)
  int dup;          // node-centred periodic: index 0 is also written to index dup (else -1)
};

// Shared-memory row layout of the column kernels.  A wavefront of shared
// memory serves 128 bytes; when a tile row (W elements) is narrower, G = 128 /
// (W sizeof(cpx<T>)) rows share a wavefront, and the row strides of the stages
// (1 for every load and for stores with Ns > 1, R for the Ns = 1 stores) would
// land them on the same banks.  Rows are then permuted within aligned groups of
// G: row i is kept in slot i ^ f(i >> lg G), f = XOR of the (lg G)-bit chunks of
// its argument.  f is linear over disjoint bit fields, and G aligned rows
// i0 + t d (d a power of two) differ in one (lg G)-bit field, so they land in G
// distinct slots.  Wide rows (G = 1) keep the padded stride W + 1.
template <typename T, int W>
struct ColRows {
  static constexpr int EB = (int)sizeof(cpx<T>);
  static constexpr int G = (W * EB >= 128) ? 1 : 128 / (W * EB);
  static_assert(G == 1 || G == 2 || G == 4, "row groups of 1, 2 or 4");
  static constexpr int LG = G == 4 ? 2 : (G == 2 ? 1 : 0);
  static constexpr int LS = G == 1 ? W + 1 : W;
  __host__ __device__ static constexpr int fold_c(int x) {
    int f = 0;
    if (G > 1)
      for (; x > 0; x >>= LG) f ^= x & (G - 1);
    return f;
  }
  // shared-memory element of natural row o, lane l, after a stage that stored to shared memory
  __device__ __forceinline__ static int at(int o, int l) {
    if constexpr (G == 1) return o * LS + l;
    else return (o ^ fold(o >> LG)) * W + l;
  }
  __device__ __forceinline__ static int fold(int x) {
    if constexpr (G == 2) {
      return __popc(x) & 1;
    } else if constexpr (G == 4) {
      x ^= x >> 16;
      x ^= x >> 8;
      x ^= x >> 4;
      x ^= x >> 2;
      return x & 3;
    } else {
      return 0;
    }
  }
};

template <typename T, int P, int W, int NT, int R, int Ns, bool INV, int SRC, int DST, bool ZIN, bool ZOUT>
__device__ __forceinline__ void xstage(cpx<T>* S, cpx<T>* v, const cpx<T>* __restrict__ tw, int tid,
                                       const ColIO<T>& io) {
  using CR = ColRows<T, W>;
  constexpr int LS = CR::LS, LG = CR::LG;
  constexpr int nbf = P / R;
  constexpr int NB = (nbf * W) / NT;
  constexpr int EPT = P * W / NT;
  static_assert(NB * R == EPT && (EPT == 16 || EPT == 32), "16 or 32 elements per thread");
  static_assert(CR::G == 1 || (nbf >= CR::G && R >= CR::G && (Ns == 1 || Ns >= CR::G)), "row permutation fields");
  constexpr int tstep = (2 * P) / (Ns * R);
  if constexpr (SRC != XS_REGS) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int idx = tid + b * NT;
      const int lane = idx % W, j = idx / W;
      // load rows j + r nbf (j < nbf): the permutation acts on j's field and r's field separately
      const int jx = j ^ CR::fold(j >> LG);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = j + r * nbf;
        if (ZIN && r >= R / 2) {
          v[b * R + r] = mk<T>((T)0, (T)0);   // zero padding: inputs at i >= P/2
        } else if constexpr (SRC == XS_SMEM) {
          if constexpr (CR::G == 1) {
            v[b * R + r] = S[i * LS + lane];
          } else {
            const int hi = r * nbf;
            v[b * R + r] = S[((jx ^ CR::fold_c(hi >> LG)) + hi) * W + lane];
          }
        } else if constexpr (SRC == XS_NAT) {
          v[b * R + r] = S[i * W + lane];
        } else {
          const int q = io.q0 + lane;
          v[b * R + r] = (q < io.npen && i < io.n_in) ? io.in[(long long)q * io.ils + (long long)i * io.ijs]
                                                      : mk<T>((T)0, (T)0);
        }
      }
    }
    // every thread has read its inputs before any thread overwrites them: needed when this stage
    // (or, from registers, the next one) writes shared memory; a last stage that stores to global
    // memory writes none
    if constexpr ((SRC == XS_SMEM || SRC == XS_NAT) && DST != XS_GLOBAL) __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int idx = tid + b * NT;
    const int j = idx / W, k = j % Ns;
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const cpx<T> w = ldg_c<T>(&tw[r * k * tstep]);
        v[b * R + r] = INV ? cmulc<T>(v[b * R + r], w) : cmul<T>(v[b * R + r], w);
      }
    }
    if constexpr (ZIN && R == 32) dft32<T, INV, true>(&v[b * R]);   // inputs 16..31 are zero padding
    else dftR<T, R, INV>(&v[b * R]);
  }
  if constexpr (DST != XS_REGS) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int idx = tid + b * NT;
      const int lane = idx % W, j = idx / W, k = j % Ns;
      const int base = (j - k) * R + k;
      // store rows base + r Ns: fields k | r Ns | (j - k) R are disjoint; for Ns = 1 the low
      // (lg G) bits come from r, otherwise from k
      const int bx = (Ns == 1) ? CR::fold(base >> LG) : (base ^ CR::fold(base >> LG));
#pragma unroll
      for (int r = 0; r < (ZOUT ? R / 2 : R); ++r) {
        const int o = base + r * Ns;
        if constexpr (DST == XS_SMEM) {
          if constexpr (CR::G == 1) {
            S[o * LS + lane] = v[b * R + r];
          } else if constexpr (Ns == 1) {
            S[(base + (r ^ CR::fold_c(r >> LG) ^ bx)) * W + lane] = v[b * R + r];
          } else {
            const int hi = r * Ns;
            S[((bx ^ CR::fold_c(hi >> LG)) + hi) * W + lane] = v[b * R + r];
          }
        } else {
          const int q = io.q0 + lane;
          if (q < io.npen) {
            if (o < io.n_out) io.out[(long long)q * io.ols + (long long)o * io.ojs] = v[b * R + r];
            if (o == 0 && io.dup >= 0) io.out[(long long)q * io.ols + (long long)io.dup * io.ojs] = v[b * R + r];
          }
        }
      }
    }
    if constexpr (DST == XS_SMEM) __syncthreads();
  }
}

template <typename T, int P, int W, bool INV, bool REV, int s, int SRC0, int DSTL, bool ZIN = false, bool ZOUT = false,
          int EPT = 16>
__device__ __forceinline__ void xstages(cpx<T>* S, cpx<T>* v, const cpx<T>* __restrict__ tw, int tid,
                                        const ColIO<T>& io) {
  constexpr int NS = ct_nstages_e(P, EPT);
  if constexpr (s < NS) {
    constexpr int R = REV ? ct_rad_rev_e(P, s, EPT) : ct_rad_e(P, s, EPT);
    constexpr int Ns = REV ? ct_ns_rev_e(P, s, EPT) : ct_ns_e(P, s, EPT);
    constexpr int SRC = s == 0 ? SRC0 : (int)XS_SMEM;
    constexpr int DST = s == NS - 1 ? DSTL : (int)XS_SMEM;
    xstage<T, P, W, P * W / EPT, R, Ns, INV, SRC, DST, ZIN && s == 0, ZOUT && s == NS - 1>(S, v, tw, tid, io);
    xstages<T, P, W, INV, REV, s + 1, SRC0, DSTL, ZIN, ZOUT, EPT>(S, v, tw, tid, io);
  }
}

// Launch order of the fused column pass along its other direction: 0, 1, n-1, 2, n-2, ... (a
// bijection of [0, n)).  Rows o and n - o read the same folded Green slice, so the CTAs that share
// it run back to back and the second read comes from L2.
__device__ __forceinline__ int mirror_order(int b, int n) {
  if (b == 0) return 0;
  const int k = (b + 1) >> 1;
  return (b & 1) ? k : n - k;
}

template <typename T>
__device__ __forceinline__ ColIO<T> col_io(const PassParams& p, int W, int n_in, int n_out, int dup, int o) {
  ColIO<T> io;
  const long long obase_i = (long long)o * p.ai.os + (long long)blockIdx.z * p.ai.cs;
  const long long obase_o = (long long)o * p.ao.os + (long long)blockIdx.z * p.ao.cs;
  io.in = (const cpx<T>*)p.in + obase_i;
  io.out = (cpx<T>*)p.out + obase_o;
  io.ils = p.ai.ls;
  io.ijs = p.ai.js;
  io.ols = p.ao.ls;
  io.ojs = p.ao.js;
  io.q0 = blockIdx.x * W;
  io.npen = p.npen;
  io.n_in = n_in;
  io.n_out = n_out;
  io.dup = dup;
  return io;
}

// Shared memory of the column kernels: the first 128-byte aligned address holds the input tile's
// mbarrier; the tile S starts 128 bytes later (the host adds 256 bytes of slack).
__device__ __forceinline__ unsigned char* col_base(unsigned char* smraw) {
  return smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u) + 128;
}

// Input tile by TMA (p.tin_rows > 0): thread 0 initialises the mbarrier (all threads must pass a
// barrier before waiting on it), then issues p.tin_rows / p.tin_box box loads of W lanes x tin_box
// rows into the dense tile S (row i of lane l at S[i W + l]); rows past the array's extent arrive
// as zeros.  p must be the kernel's __grid_constant__ parameter (the map is read in place).
template <typename T, int W>
__device__ __forceinline__ void tile_tma_issue(const PassParams& p, cpx<T>* S, unsigned long long* bar, int o) {
  constexpr int U = (int)sizeof(cpx<T>) / 8;  // 8-byte units per element
  const int q0 = blockIdx.x * W, c = blockIdx.z;
  mbar_expect_tx(bar, (unsigned)((size_t)p.tin_rows * W * sizeof(cpx<T>)));
  for (int r0 = 0; r0 < p.tin_rows; r0 += p.tin_box) {
    if (p.axis == 1) tma_load_4d(S + (size_t)r0 * W, &p.tin, q0 * U, r0, o, c, bar);
    else tma_load_4d(S + (size_t)r0 * W, &p.tin, q0 * U, o, r0, c, bar);
  }
}

template <typename T, int PC, int WC, bool HZ, int EPT = 16>
__global__ void __launch_bounds__(ColBounds<T, PC, WC, EPT>::threads, ColBounds<T, PC, WC, EPT>::minb)
    k_fwd_c2c_col(const __grid_constant__ PassParams p) {
  pass_entry(p);
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned char* base = col_base(smraw);
  unsigned long long* mbar_in = reinterpret_cast<unsigned long long*>(base - 128);
  cpx<T>* S = reinterpret_cast<cpx<T>*>(base);
  cpx<T> v[EPT];
  const int tid = threadIdx.x;
  ColIO<T> io = col_io<T>(p, WC, p.n_use, PC, -1, blockIdx.y);
  const cpx<T>* tw = (const cpx<T>*)p.tw;
  if (p.tin_rows) {
    if (tid == 0) mbar_init(mbar_in, 1);
    __syncthreads();
    if (tid == 0) tile_tma_issue<T, WC>(p, S, mbar_in, blockIdx.y);
    if (!mbar_wait_bounded(mbar_in, p.errflag, 2, p.dbg_wait & 2)) io.npen = 0;  // no stores of a partial tile
    xstages<T, PC, WC, false, false, 0, XS_NAT, XS_GLOBAL, HZ, false, EPT>(S, v, tw, tid, io);
  } else {
    xstages<T, PC, WC, false, false, 0, XS_GLOBAL, XS_GLOBAL, HZ, false, EPT>(S, v, tw, tid, io);
  }
}

template <typename T, int PC, int WC, bool HZ, int EPT = 16>
__global__ void __launch_bounds__(ColBounds<T, PC, WC, EPT>::threads, ColBounds<T, PC, WC, EPT>::minb)
    k_inv_c2c_col(const __grid_constant__ PassParams p) {
  pass_entry(p);
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned char* base = col_base(smraw);
  unsigned long long* mbar_in = reinterpret_cast<unsigned long long*>(base - 128);
  cpx<T>* S = reinterpret_cast<cpx<T>*>(base);
  cpx<T> v[EPT];
  const int tid = threadIdx.x;
  const int dup = (p.type == T_PER && p.center == C_NODE && p.n_data > p.N) ? p.N : -1;
  ColIO<T> io = col_io<T>(p, WC, PC, p.n_data, dup, blockIdx.y);
  const cpx<T>* tw = (const cpx<T>*)p.tw;
  if (p.tin_rows) {
    if (tid == 0) mbar_init(mbar_in, 1);
    __syncthreads();
    if (tid == 0) tile_tma_issue<T, WC>(p, S, mbar_in, blockIdx.y);
    if (!mbar_wait_bounded(mbar_in, p.errflag, 2, p.dbg_wait & 2)) io.npen = 0;
    xstages<T, PC, WC, true, false, 0, XS_NAT, XS_GLOBAL, false, HZ, EPT>(S, v, tw, tid, io);
  } else {
    xstages<T, PC, WC, true, false, 0, XS_GLOBAL, XS_GLOBAL, false, HZ, EPT>(S, v, tw, tid, io);
  }
}

template <typename T, int PC, int WC, bool HZ, int EPT = 16>
__global__ void __launch_bounds__(ColBounds<T, PC, WC, EPT>::threads, ColBounds<T, PC, WC, EPT>::minb)
    k_fused_c2c_col(const __grid_constant__ PassParams p) {
  pass_entry(p);
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int P = PC, W = WC, NT = PC * WC / EPT;
  unsigned char* base = col_base(smraw);
  unsigned long long* mbar_in = reinterpret_cast<unsigned long long*>(base - 128);
  unsigned long long* mbar_g = mbar_in + 1;
  cpx<T>* S = reinterpret_cast<cpx<T>*>(base);
  long long* goff = reinterpret_cast<long long*>(base + (size_t)P * (W + 1) * sizeof(cpx<T>));
  T* k2p = reinterpret_cast<T*>(goff + W);
  // stored spectrum slice of this tile, W lanes x (P/2 + 1) folded modes (p.gpre), at a 128-byte
  // aligned shared address (the host adds the slack)
  unsigned char* graw = base + (size_t)P * (W + 1) * sizeof(cpx<T>) + (size_t)W * (sizeof(long long) + sizeof(T));
  T* Gs = reinterpret_cast<T*>(graw + ((128u - (smem_u32(graw) & 127u)) & 127u));
  constexpr int GH = P / 2 + 1;
  const int tid = threadIdx.x;
  const int q0 = blockIdx.x * W;
  const int o = mirror_order(blockIdx.y, gridDim.y);
  const bool tma_g = p.gpre && p.gmap;
  // TMA copies: the input tile (p.tin_rows) and the Green slice (p.gmap), each completed on its
  // own mbarrier; thread 0 initialises both before the CTA barrier and then issues the loads
  if (p.tin_rows || tma_g) {
    if (tid == 0) {
      if (p.tin_rows) mbar_init(mbar_in, 1);
      if (tma_g) mbar_init(mbar_g, 1);
    }
    __syncthreads();
    if (tid == 0) {
      if (p.tin_rows) tile_tma_issue<T, W>(p, S, mbar_in, o);
      if (tma_g) {
        const FusedGreen& g = p.g;
        const int nd = p.axis == 2 ? 1 : 2;  // the direction o runs along
        const int go = g.fold[nd] ? min(o, g.fold[nd] - o) : o;
        const char* maps = (const char*)p.gmap;
        mbar_expect_tx(mbar_g, (unsigned)(GH * W * sizeof(T)));
        for (int r0 = 0; r0 < P / 2; r0 += p.gbox) {
          if (p.axis == 2) tma_load_3d(Gs + (size_t)r0 * W, maps, q0, go, r0, mbar_g);
          else tma_load_3d(Gs + (size_t)r0 * W, maps, q0, r0, go, mbar_g);
        }
        if (p.axis == 2) tma_load_3d(Gs + (size_t)(P / 2) * W, maps + 128, q0, go, P / 2, mbar_g);
        else tma_load_3d(Gs + (size_t)(P / 2) * W, maps + 128, q0, P / 2, go, mbar_g);
      }
    }
  }
  if (p.gpre && !tma_g) {
    // asynchronous copy (cp.async) of the Green slice, overlapped with the forward transform;
    // NT is a multiple of W, so each thread serves one lane
    const int lane = tid % W;
    long long go;
    T kp;
    pencil_green_base<T>(p, q0 + lane, o, &go, &kp);
    if (q0 + lane < p.npen) {
      const long long st3 = p.axis == 1 ? (long long)p.g.gpitch : (long long)p.g.gpitch * p.g.gext[1];
      const T* src = (const T*)p.g.stored + go;
      for (int g3 = tid / W; g3 < GH; g3 += NT / W) cp_async_elem<sizeof(T)>(&Gs[g3 * W + lane], src + g3 * st3);
    }
    cp_async_commit();
  } else if (!p.gpre) {
    for (int lane = tid; lane < W; lane += NT) pencil_green_base<T>(p, q0 + lane, o, &goff[lane], &k2p[lane]);
  }
  const int dup = (p.type == T_PER && p.center == C_NODE && p.n_data > p.N) ? p.N : -1;
  ColIO<T> io = col_io<T>(p, W, p.n_use, p.n_data, dup, o);
  const cpx<T>* tw = (const cpx<T>*)p.tw;
  cpx<T> v[EPT];
  // forward: HBM (or the TMA tile) -> ... -> registers (the first stage's barrier also publishes goff/k2p)
  if (p.tin_rows) {
    if (!mbar_wait_bounded(mbar_in, p.errflag, 2, p.dbg_wait & 2)) io.npen = 0;
    xstages<T, P, W, false, false, 0, XS_NAT, XS_REGS, HZ, false, EPT>(S, v, tw, tid, io);
  } else {
    xstages<T, P, W, false, false, 0, XS_GLOBAL, XS_REGS, HZ, false, EPT>(S, v, tw, tid, io);
  }
  // u^ = G^ f^ on the EPT elements this thread holds: indices j + r P/RL
  constexpr int RL = ct_rad_e(P, ct_nstages_e(P, EPT) - 1, EPT);
  constexpr int NB = EPT / RL;
  if (p.gpre) {
    if (tma_g) {
      if (!mbar_wait_bounded(mbar_g, p.errflag, 1, p.dbg_wait & 1)) io.npen = 0;
    } else {
      cp_async_wait_all();
      __syncthreads();
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int idx = tid + b * NT;
      const int lane = idx % W, j = idx / W;
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int k = j + r * (P / RL);
        v[b * RL + r] = cscale<T>(v[b * RL + r], Gs[min(k, P - k) * W + lane]);
      }
    }
  } else {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int idx = tid + b * NT;
      const int lane = idx % W, j = idx / W;
      const long long go = goff[lane];
      const T kp = k2p[lane];
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int k = j + r * (P / RL);
        const T G = green_at<T>(p, go, kp, min(k, P - k));
        v[b * RL + r] = cscale<T>(v[b * RL + r], G);
      }
    }
  }
  // inverse, radices in reverse order: registers -> ... -> HBM
  xstages<T, P, W, true, true, 0, XS_REGS, XS_GLOBAL, false, HZ, EPT>(S, v, tw, tid, io);
}

// ---------------------------------------------------------------------------
// Row-mode passes (x, contiguous in memory) of real data on the column kernels' register-chained
// stages, for the periodic and the doubled unbounded cell-centred directions (R2C modes):
// the CTA's 2W rows are placed as W lanes of packed pairs (row q0 + 2l in the real part, row
// q0 + 2l + 1 in the imaginary part) in the dense tile the first stage reads, the stages run as in
// the column kernels, and the modes are split and stored with the lane index fastest, so that
// a warp touches W lanes of a few consecutive rows of the tile (no bank conflicts) and a few
// consecutive modes of each of 2W rows in memory (whole sectors).
// ---------------------------------------------------------------------------
template <typename T, int PC, int WC, bool HZ, int EPT>
__global__ void __launch_bounds__(ColBounds<T, PC, WC, EPT>::threads, ColBounds<T, PC, WC, EPT>::minb)
    k_fwd_rowx(const __grid_constant__ PassParams p) {
  pass_entry(p);
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int P = PC, W = WC, NT = PC * WC / EPT;
  using CR = ColRows<T, W>;
  cpx<T>* S = reinterpret_cast<cpx<T>*>(col_base(smraw));
  const int tid = threadIdx.x;
  const int q0 = blockIdx.x * 2 * W;
  const T* in = (const T*)p.in + (long long)blockIdx.z * p.ai.cs;
  cpx<T>* out = (cpx<T>*)p.out + (long long)blockIdx.z * p.ao.cs;
  const int nd = p.n_use;  // P/2 values then zero padding (doubled), or P (periodic)
  // S[i W + l] = (row q0 + 2l, row q0 + 2l + 1) at position i, lane index fastest: a warp writes
  // consecutive tile elements and reads a few consecutive values of each of its rows; the loads of
  // U iterations are issued before any is used: all of a thread's (EPT, or EPT/2 with the zero
  // half) where the kernel has 128 registers, 8 in the 64-register FP32 kernels
  constexpr int U = (sizeof(T) > 4 || EPT == 32) ? (HZ ? EPT / 2 : EPT) : 8;
  const int tot = W * nd;
  for (int base = tid; base < tot; base += U * NT) {
    T a[U], b[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * NT;
      const int l = idx % W, i = idx / W;
      const int qa = q0 + 2 * l;
      const long long off = (long long)qa * p.ai.ls + i;
      a[u] = (idx < tot && qa < p.npen) ? ld_real<T>(in, off, p.in_f64) : (T)0;
      b[u] = (idx < tot && qa + 1 < p.npen) ? ld_real<T>(in, off + p.ai.ls, p.in_f64) : (T)0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * NT;
      if (idx < tot) S[(idx / W) * W + idx % W] = mk<T>(a[u], b[u]);
    }
  }
  __syncthreads();
  ColIO<T> io{};
  cpx<T> v[EPT];
  xstages<T, P, W, false, false, 0, XS_NAT, XS_SMEM, HZ, false, EPT>(S, v, (const cpx<T>*)p.tw, tid, io);
  // modes k = 0 .. P/2 of every lane, split into the two packed rows (Hermitian symmetry)
  constexpr int NM = P / 2 + 1;
  for (int idx = tid; idx < W * NM; idx += NT) {
    const int l = idx % W, k = idx / W;
    const cpx<T> zk = S[CR::at(k, l)], zm = S[CR::at(k == 0 ? 0 : P - k, l)];
    const int qa = q0 + 2 * l;
    if (qa < p.npen) out[(long long)qa * p.ao.ls + k] = split<T>(zk, zm, 0);
    if (qa + 1 < p.npen) out[(long long)(qa + 1) * p.ao.ls + k] = split<T>(zk, zm, 1);
  }
}

template <typename T, int PC, int WC, bool HZ, int EPT>
__global__ void __launch_bounds__(ColBounds<T, PC, WC, EPT>::threads, ColBounds<T, PC, WC, EPT>::minb)
    k_inv_rowx(const __grid_constant__ PassParams p) {
  pass_entry(p);
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int P = PC, W = WC, NT = PC * WC / EPT;
  using CR = ColRows<T, W>;
  cpx<T>* S = reinterpret_cast<cpx<T>*>(col_base(smraw));
  const int tid = threadIdx.x;
  const int q0 = blockIdx.x * 2 * W;
  const cpx<T>* in = (const cpx<T>*)p.in + (long long)blockIdx.z * p.ai.cs;
  T* out = (T*)p.out + (long long)blockIdx.z * p.ao.cs;
  // with p.rows_bulk the CTA's 2W input rows (contiguous in memory) first arrive by one bulk copy
  const cpx<T>* rows = in + (long long)q0 * p.ai.ls;
  if (p.rows_bulk) {
    unsigned char* sb = smraw + p.rows_off;
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(sb) - 16;
    const int nrows = min(2 * W, p.npen - q0);
    if (tid == 0) mbar_init(bar, 1);
    __syncthreads();
    if (tid == 0) {
      const unsigned bytes = (unsigned)((size_t)nrows * p.ai.ls * sizeof(cpx<T>));
      mbar_expect_tx(bar, bytes);
      bulk_load(sb, rows, bytes, bar);
    }
    const bool ok = mbar_wait_bounded(bar, p.errflag, 2, p.dbg_wait & 2);
    if (__syncthreads_or(!ok)) return;  // the tile's input did not arrive in time: no stores
    rows = reinterpret_cast<const cpx<T>*>(sb);
  }
  // modes of the two packed rows of every lane -> Z_k = A_k + i B_k and Z_{P-k} = conj(A_k) + i conj(B_k);
  // the loads of U iterations are issued before any is used
  constexpr int NM = P / 2 + 1, U = 4;
  for (int base = tid; base < W * NM; base += U * NT) {
    cpx<T> A[U], B[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * NT;
      const int l = idx % W, k = idx / W;
      const int qa = q0 + 2 * l;
      A[u] = mk<T>((T)0, (T)0);
      B[u] = A[u];
      if (idx < W * NM) {
        if (qa < p.npen) A[u] = rows[(long long)(2 * l) * p.ai.ls + k];
        if (qa + 1 < p.npen) B[u] = rows[(long long)(2 * l + 1) * p.ai.ls + k];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * NT;
      if (idx >= W * NM) continue;
      const int l = idx % W, k = idx / W;
      if (k == 0 || k == P / 2) {  // DC and Nyquist of a real signal are real
        A[u].y = (T)0;
        B[u].y = (T)0;
      }
      S[k * W + l] = mk<T>(A[u].x - B[u].y, A[u].y + B[u].x);
      if (k != 0 && k != P / 2) S[(P - k) * W + l] = mk<T>(A[u].x + B[u].y, B[u].x - A[u].y);
    }
  }
  __syncthreads();
  ColIO<T> io{};
  cpx<T> v[EPT];
  xstages<T, P, W, true, false, 0, XS_NAT, XS_SMEM, false, HZ, EPT>(S, v, (const cpx<T>*)p.tw, tid, io);
  // data positions i < n_data of both packed rows
  const int nd = p.n_data;
  for (int idx = tid; idx < W * nd; idx += NT) {
    const int l = idx % W, i = idx / W;
    const cpx<T> z = S[CR::at(i, l)];
    const int qa = q0 + 2 * l;
    const long long off = (long long)qa * p.ao.ls + i;
    if (qa < p.npen) st_real<T>(out, off, z.x, p.out_f64);
    if (qa + 1 < p.npen) st_real<T>(out, off + p.ao.ls, z.y, p.out_f64);
  }
}

// ---------------------------------------------------------------------------
// Instantiation helpers: one launcher and one smem-limit setter per <T, PC, WC>.
// ---------------------------------------------------------------------------
// Column kernels with radix-32 stages (32 elements per thread) are compiled for FP32 at P = 1024
// (the planner uses them for the fused pass).
template <typename T, int PC> constexpr bool has_ept32() { return std::is_same<T, float>::value && PC == 1024; }

// Launch a pass kernel; with p.pdl as a programmatic dependent of the stream's previous kernel.
template <typename K>
cudaError_t pass_launch(K kernel, const PassParams& p, dim3 grid, int nthr, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3((unsigned)nthr);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = p.pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, p);
}

template <typename T, int PC, int WC, bool HZ>
cudaError_t launch_kind_hz(int kind, const PassParams& p, dim3 grid, int nthr, size_t smem, cudaStream_t st) {
  if constexpr (PC > 0 && (std::is_same<T, float>::value || std::is_same<T, dfloat>::value)) {
    if (p.axis == 0 && p.rowx && (kind == K_FWD_REAL || kind == K_INV_REAL)) {
      const bool fwd = kind == K_FWD_REAL;
      if constexpr (has_ept32<T, PC>()) {
        if (p.ept == 32) {
          if (fwd) return pass_launch(k_fwd_rowx<T, PC, WC, HZ, 32>, p, grid, nthr, smem, st);
          else return pass_launch(k_inv_rowx<T, PC, WC, HZ, 32>, p, grid, nthr, smem, st);
          return cudaGetLastError();
        }
      }
      if (fwd) return pass_launch(k_fwd_rowx<T, PC, WC, HZ, 16>, p, grid, nthr, smem, st);
      else return pass_launch(k_inv_rowx<T, PC, WC, HZ, 16>, p, grid, nthr, smem, st);
      return cudaGetLastError();
    }
  }
  if constexpr (PC > 0) {
    if constexpr (has_ept32<T, PC>()) {
      if (p.axis != 0 && p.ept == 32) {
        switch (kind) {
          case K_FWD_C2C: return pass_launch(k_fwd_c2c_col<T, PC, WC, HZ, 32>, p, grid, nthr, smem, st);
          case K_INV_C2C: return pass_launch(k_inv_c2c_col<T, PC, WC, HZ, 32>, p, grid, nthr, smem, st);
          case K_FUSED_C2C: return pass_launch(k_fused_c2c_col<T, PC, WC, HZ, 32>, p, grid, nthr, smem, st);
          default: break;
        }
      }
    }
    if (p.axis != 0) {  // column passes of complex data: register-chained kernels
      switch (kind) {
        case K_FWD_C2C: return pass_launch(k_fwd_c2c_col<T, PC, WC, HZ>, p, grid, nthr, smem, st);
        case K_INV_C2C: return pass_launch(k_inv_c2c_col<T, PC, WC, HZ>, p, grid, nthr, smem, st);
        case K_FUSED_C2C: return pass_launch(k_fused_c2c_col<T, PC, WC, HZ>, p, grid, nthr, smem, st);
        default: break;
      }
    }
  }
  switch (kind) {
    case K_FWD_REAL: return pass_launch(k_fwd_real<T, PC, WC, HZ>, p, grid, nthr, smem, st);
    case K_INV_REAL: return pass_launch(k_inv_real<T, PC, WC, HZ>, p, grid, nthr, smem, st);
    case K_FWD_C2C: return pass_launch(k_fwd_c2c<T, PC, WC, HZ>, p, grid, nthr, smem, st);
    case K_INV_C2C: return pass_launch(k_inv_c2c<T, PC, WC, HZ>, p, grid, nthr, smem, st);
    case K_FUSED_REAL: return pass_launch(k_fused_real<T, PC, WC, HZ>, p, grid, nthr, smem, st);
    case K_FUSED_C2C: return pass_launch(k_fused_c2c<T, PC, WC, HZ>, p, grid, nthr, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

// p.hz: the pass's transform is a cell-centred doubled (unbounded) one -- half of its
// input is zero padding and half of its output is discarded (compile-time engine only)
template <typename T, int PC, int WC>
cudaError_t launch_kind(int kind, const PassParams& p, dim3 grid, int nthr, size_t smem, cudaStream_t st) {
  if constexpr (PC > 0) {
    if (p.hz) return launch_kind_hz<T, PC, WC, true>(kind, p, grid, nthr, smem, st);
  }
  return launch_kind_hz<T, PC, WC, false>(kind, p, grid, nthr, smem, st);
}

template <typename T, int PC, int WC, bool HZ>
cudaError_t set_limits_hz() {
  const int lim = 227 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_fwd_real<T, PC, WC, HZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_inv_real<T, PC, WC, HZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_fwd_c2c<T, PC, WC, HZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_inv_c2c<T, PC, WC, HZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_fused_real<T, PC, WC, HZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if constexpr (PC > 0) {
    if ((e = cudaFuncSetAttribute(k_fwd_c2c_col<T, PC, WC, HZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(k_inv_c2c_col<T, PC, WC, HZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(k_fused_c2c_col<T, PC, WC, HZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if constexpr (std::is_same<T, float>::value || std::is_same<T, dfloat>::value) {
      if ((e = cudaFuncSetAttribute(k_fwd_rowx<T, PC, WC, HZ, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
      if ((e = cudaFuncSetAttribute(k_inv_rowx<T, PC, WC, HZ, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
      if constexpr (has_ept32<T, PC>()) {
        if ((e = cudaFuncSetAttribute(k_fwd_rowx<T, PC, WC, HZ, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
        if ((e = cudaFuncSetAttribute(k_inv_rowx<T, PC, WC, HZ, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
      }
    }
    if constexpr (has_ept32<T, PC>()) {
      if ((e = cudaFuncSetAttribute(k_fwd_c2c_col<T, PC, WC, HZ, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
      if ((e = cudaFuncSetAttribute(k_inv_c2c_col<T, PC, WC, HZ, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
      if ((e = cudaFuncSetAttribute(k_fused_c2c_col<T, PC, WC, HZ, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    }
  }
  return cudaFuncSetAttribute(k_fused_c2c<T, PC, WC, HZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

template <typename T, int PC, int WC>
cudaError_t set_limits_kind() {
  cudaError_t e = set_limits_hz<T, PC, WC, false>();
  if constexpr (PC > 0) {
    if (!e) e = set_limits_hz<T, PC, WC, true>();
  }
  return e;
}

}  // namespace flups
