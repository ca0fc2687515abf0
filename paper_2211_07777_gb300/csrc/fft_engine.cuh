// Shared-memory FFT engine for one tile of pencils (sm_103a).
//
// A tile holds W "lanes" of one complex sequence of length P each, laid out in
// shared memory as S[j * LS + lane] (j = sequence index, LS >= W).  The
// transform is a Stockham auto-sort FFT of P = 2^a 3^b in radix-16/8/4/2/3
// stages; every stage reads its butterfly inputs from one shared buffer into
// registers, applies the inter-stage twiddles and a register radix-R DFT, and
// writes the outputs in natural order to the other buffer.  Twiddles
// come from a table of exp(-2 pi i m / (2P)), m = 0 .. 2P-1, generated in FP64
// on the host and rounded once to the path precision.
//
// The method's 1D transforms (Section "Methodology", eq. of Section 2.2: DFT,
// DCT/DST I-IV through their periodic extensions) all reduce to this complex
// FFT of the extended sequence.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "dfloat.cuh"

namespace flups {

template <typename T> struct cpx_t;
template <> struct cpx_t<float> { using type = float2; };
template <> struct cpx_t<double> { using type = double2; };
template <> struct cpx_t<dfloat> { using type = cdfloat; };
template <typename T> using cpx = typename cpx_t<T>::type;

// read-only cached loads (the double-float types go through their vector twins)
template <typename T> __device__ __forceinline__ cpx<T> ldg_c(const cpx<T>* p) { return __ldg(p); }
template <> __device__ __forceinline__ cdfloat ldg_c<dfloat>(const cdfloat* p) {
  const float4 q = __ldg(reinterpret_cast<const float4*>(p));
  cdfloat c;
  c.x = dfloat(q.x, q.y);
  c.y = dfloat(q.z, q.w);
  return c;
}
// Asynchronous global -> shared copy of one element (4 or 8 bytes, cp.async through L1),
// completed by cp_async_wait_all() in the same thread (plus a barrier for other readers).
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* dst_smem, const void* src) {
  static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Tensor-memory-accelerator (TMA) copies completed through a shared-memory mbarrier.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 4D tile load of the box at coordinates (c0, c1, c2, c3) of the tensor map into shared memory
__device__ __forceinline__ void tma_load_4d(void* dst, const void* tmap, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];\n" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Time limits of a bounded mbarrier wait: the copies it waits for take microseconds, so a wait
// that has not completed after kWaitLimitNs is declared failed; the kernel then waits at most
// kDrainLimitNs more for the copies still in flight (so that no copy writes into the shared memory
// of a CTA that has exited) and skips its global stores.  Once a failure has been recorded, later
// waits are given kGraceNs only instead of the full limit, so that a solve whose copies never
// arrive ends quickly.
constexpr unsigned long long kWaitLimitNs = 1000000000ull;   // 1 s
constexpr unsigned long long kGraceNs = 1000000ull;          // 1 ms
constexpr unsigned long long kDrainLimitNs = 100000000ull;   // 0.1 s
// Bounded wait for phase 0 of an mbarrier.  Returns true when the copies completed within the
// limit; otherwise records `code` in *errflag (when non-null and still 0: the first code recorded
// is kept), drains as above and returns false (the tile's data are then not valid).  force_fail
// (a test hook) makes the first limit zero: the wait gives up at once and only the drain waits for
// the copies, which do complete.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, int* errflag, int code,
                                                  bool force_fail = false) {
  if (!force_fail && mbar_try_wait(bar, 0)) return true;
  bool done = false;
  unsigned long long limit = kWaitLimitNs;
  if (force_fail) limit = 0;
  else if (errflag && *(volatile int*)errflag != 0) limit = kGraceNs;
  const unsigned long long t0 = global_ns();
  while (!done && global_ns() - t0 < limit) done = mbar_try_wait(bar, 0);
  if (done) return true;
  if (errflag) atomicCAS(errflag, 0, code);
  const unsigned long long t1 = global_ns();
  while (!done && global_ns() - t1 < kDrainLimitNs) done = mbar_try_wait(bar, 0);
  return false;
}
// 1D bulk copy of `bytes` contiguous bytes from global to shared memory, completed on an mbarrier
// (both addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// 3D tile load of the box at coordinates (c0, c1, c2) of the tensor map into shared memory
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int c0, int c1, int c2,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

template <typename T> __device__ __forceinline__ T ldg_r(const T* p) { return __ldg(p); }
template <> __device__ __forceinline__ dfloat ldg_r<dfloat>(const dfloat* p) {
  const float2 q = __ldg(reinterpret_cast<const float2*>(p));
  return dfloat(q.x, q.y);
}

template <typename T> __host__ __device__ __forceinline__ cpx<T> mk(T re, T im) { cpx<T> c; c.x = re; c.y = im; return c; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __host__ __device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __host__ __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T> __host__ __device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T> __host__ __device__ __forceinline__ cpx<T> cconj(cpx<T> a) { return mk<T>(a.x, -a.y); }
template <typename T> __host__ __device__ __forceinline__ cpx<T> cscale(cpx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV> __host__ __device__ __forceinline__ cpx<T> mul_mi(cpx<T> a) {
  return INV ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

// ---------------------------------------------------------------------------
// Register DFTs of radix 2, 3, 4, 8, 16 (forward: exp(-2 pi i q r / R)).
// The constants are the exact values cos(pi/4), cos(pi/8), sin(pi/8), sqrt(3)/2.
// ---------------------------------------------------------------------------
template <typename T, bool INV> __host__ __device__ __forceinline__ void dft2(cpx<T>& a, cpx<T>& b) {
  cpx<T> t = a; a = cadd<T>(t, b); b = csub<T>(t, b);
}

template <typename T, bool INV> __host__ __device__ __forceinline__ void dft4(cpx<T>& a, cpx<T>& b, cpx<T>& c, cpx<T>& d) {
  cpx<T> t0 = cadd<T>(a, c), t1 = csub<T>(a, c), t2 = cadd<T>(b, d), t3 = mul_mi<T, INV>(csub<T>(b, d));
  a = cadd<T>(t0, t2); c = csub<T>(t0, t2); b = cadd<T>(t1, t3); d = csub<T>(t1, t3);
}

template <typename T, bool INV> __host__ __device__ __forceinline__ void dft3(cpx<T>& a, cpx<T>& b, cpx<T>& c) {
  const T s3 = (T)0.86602540378443864676372317075294;
  cpx<T> t1 = cadd<T>(b, c);
  cpx<T> t2 = mk<T>(a.x - (T)0.5 * t1.x, a.y - (T)0.5 * t1.y);
  cpx<T> t3 = mul_mi<T, INV>(cscale<T>(csub<T>(b, c), s3));
  a = cadd<T>(a, t1); b = cadd<T>(t2, t3); c = csub<T>(t2, t3);
}

// rotate by W8^1 = (1 - i)/sqrt2 (forward) or its conjugate
template <typename T, bool INV> __host__ __device__ __forceinline__ cpx<T> rot8_1(cpx<T> a) {
  const T r = (T)0.70710678118654752440084436210485;
  return INV ? mk<T>(r * (a.x - a.y), r * (a.x + a.y)) : mk<T>(r * (a.x + a.y), r * (a.y - a.x));
}
// rotate by W8^3 = (-1 - i)/sqrt2 (forward) or its conjugate
template <typename T, bool INV> __host__ __device__ __forceinline__ cpx<T> rot8_3(cpx<T> a) {
  const T r = (T)0.70710678118654752440084436210485;
  return INV ? mk<T>(-r * (a.x + a.y), r * (a.x - a.y)) : mk<T>(r * (a.y - a.x), -r * (a.x + a.y));
}

template <typename T, bool INV> __host__ __device__ __forceinline__ void dft8(cpx<T>* v) {
  // radix-2 DIT on top of two radix-4 DFTs
  cpx<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  cpx<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<T, INV>(e0, e1, e2, e3);
  dft4<T, INV>(o0, o1, o2, o3);
  o1 = rot8_1<T, INV>(o1);
  o2 = mul_mi<T, INV>(o2);
  o3 = rot8_3<T, INV>(o3);
  v[0] = cadd<T>(e0, o0); v[4] = csub<T>(e0, o0);
  v[1] = cadd<T>(e1, o1); v[5] = csub<T>(e1, o1);
  v[2] = cadd<T>(e2, o2); v[6] = csub<T>(e2, o2);
  v[3] = cadd<T>(e3, o3); v[7] = csub<T>(e3, o3);
}

template <typename T, bool INV> __host__ __device__ __forceinline__ cpx<T> tw16(cpx<T> a, int m) {
  // multiply by W16^m, m in [0, 9]
  const T c1 = (T)0.92387953251128675612818318939679;   // cos(pi/8)
  const T s1 = (T)0.38268343236508977172845998403040;   // sin(pi/8)
  const T r = (T)0.70710678118654752440084436210485;
  T c, s;  // W16^m = c - i s (forward)
  switch (m) {
    case 0: return a;
    case 1: c = c1; s = s1; break;
    case 2: c = r; s = r; break;
    case 3: c = s1; s = c1; break;
    case 4: return mul_mi<T, INV>(a);
    case 6: c = -r; s = r; break;
    case 9: c = -c1; s = -s1; break;
    default: c = (T)0; s = (T)0; break;
  }
  if (INV) s = -s;
  return mk<T>(a.x * c + a.y * s, a.y * c - a.x * s);
}

template <typename T, bool INV> __host__ __device__ __forceinline__ void dft16(cpx<T>* v) {
  // 4 x 4: columns n2 = 0..3 hold x[4 n1 + n2]
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<T, INV>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
  // now v[4 k1 + n2] = Y[n2][k1]; twiddle by W16^(n2 k1)
  v[5] = tw16<T, INV>(v[5], 1);
  v[6] = tw16<T, INV>(v[6], 2);
  v[7] = tw16<T, INV>(v[7], 3);
  v[9] = tw16<T, INV>(v[9], 2);
  v[10] = tw16<T, INV>(v[10], 4);
  v[11] = tw16<T, INV>(v[11], 6);
  v[13] = tw16<T, INV>(v[13], 3);
  v[14] = tw16<T, INV>(v[14], 6);
  v[15] = tw16<T, INV>(v[15], 9);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<T, INV>(v[4 * k1 + 0], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  // v[4 k1 + k2] = X[k1 + 4 k2]: transpose the 4 x 4 index
  cpx<T> t[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[4 * k1 + k2];
}

// cos(pi m / 16) for any integer m, from the exact first-octant values
// cos(0, pi/16, pi/8, 3pi/16, pi/4) and sin(3pi/16, pi/8, pi/16) (= cos of 5pi/16, 3pi/8, 7pi/16).
__host__ __device__ constexpr double cos_pi16_octant(int m) {  // 0 <= m <= 8
  return m == 0 ? 1.0
       : m == 1 ? 0.980785280403230449126182236134239
       : m == 2 ? 0.9238795325112867561281831893967883
       : m == 3 ? 0.8314696123025452370787883776179058
       : m == 4 ? 0.707106781186547524400844362104849
       : m == 5 ? 0.5555702330196022247428308139485329
       : m == 6 ? 0.3826834323650897717284599840303989
       : m == 7 ? 0.1950903220161282678482848684770222
       : 0.0;
}
__host__ __device__ constexpr double cos_pi16(int m) {
  int r = ((m % 32) + 32) % 32;  // period 32
  if (r > 16) r = 32 - r;        // even
  return r > 8 ? -cos_pi16_octant(16 - r) : cos_pi16_octant(r);
}

// multiply by W32^M = exp(-2 pi i M / 32) (forward) or its conjugate, M a compile-time constant
template <typename T, bool INV, int M> __host__ __device__ __forceinline__ cpx<T> tw32(cpx<T> a) {
  constexpr int m = M & 31;
  if constexpr (m == 0) {
    return a;
  } else if constexpr (m == 8) {
    return mul_mi<T, INV>(a);
  } else if constexpr (m == 16) {
    return mk<T>(-a.x, -a.y);
  } else if constexpr (m == 24) {
    return mul_mi<T, !INV>(a);
  } else {
    constexpr double c = cos_pi16(m), sn = cos_pi16(8 - m);  // W32^m = c - i sn
    const T cc = (T)c, s = INV ? (T)(-sn) : (T)sn;
    return mk<T>(a.x * cc + a.y * s, a.y * cc - a.x * s);
  }
}

// DFT-4 of (a, b, 0, 0): the upper half of the inputs is zero padding
template <typename T, bool INV> __host__ __device__ __forceinline__ void dft4_half(cpx<T>& a, cpx<T>& b, cpx<T>& c,
                                                                                  cpx<T>& d) {
  const cpx<T> t3 = mul_mi<T, INV>(b);
  c = csub<T>(a, b);
  d = csub<T>(a, t3);
  const cpx<T> a0 = a;
  a = cadd<T>(a0, b);
  b = cadd<T>(a0, t3);
}

template <typename T, bool INV, int K1, int N2> __host__ __device__ __forceinline__ void dft32_twiddle(cpx<T>* v) {
  if constexpr (N2 < 8) {
    v[8 * K1 + N2] = tw32<T, INV, N2 * K1>(v[8 * K1 + N2]);
    dft32_twiddle<T, INV, K1, N2 + 1>(v);
  }
}

// DFT-32 in registers as 4 x 8: inputs x[8 n1 + n2]; a DFT-4 over n1 for every n2 (ZH: the
// inputs 16..31 are zero padding), twiddles W32^(n2 k1), a DFT-8 over n2 for every k1, which
// leaves X[k1 + 4 k2] in v[8 k1 + k2]; the index is then transposed to natural order.
template <typename T, bool INV, bool ZH = false> __host__ __device__ __forceinline__ void dft32(cpx<T>* v) {
#pragma unroll
  for (int n2 = 0; n2 < 8; ++n2) {
    if constexpr (ZH) dft4_half<T, INV>(v[n2], v[8 + n2], v[16 + n2], v[24 + n2]);
    else dft4<T, INV>(v[n2], v[8 + n2], v[16 + n2], v[24 + n2]);
  }
  dft32_twiddle<T, INV, 1, 1>(v);
  dft32_twiddle<T, INV, 2, 1>(v);
  dft32_twiddle<T, INV, 3, 1>(v);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft8<T, INV>(&v[8 * k1]);
  cpx<T> t[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) t[i] = v[i];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) v[k1 + 4 * k2] = t[8 * k1 + k2];
}

template <typename T, int R, bool INV> __host__ __device__ __forceinline__ void dftR(cpx<T>* v) {
  if constexpr (R == 2) dft2<T, INV>(v[0], v[1]);
  else if constexpr (R == 3) dft3<T, INV>(v[0], v[1], v[2]);
  else if constexpr (R == 4) dft4<T, INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<T, INV>(v);
  else if constexpr (R == 16) dft16<T, INV>(v);
  else if constexpr (R == 32) dft32<T, INV>(v);
}

// ---------------------------------------------------------------------------
// One Stockham stage over the whole tile, from buffer X to buffer Y (ping-pong:
// no thread has to hold more than one butterfly, whatever the tile size).
// ---------------------------------------------------------------------------
template <typename T, int R, bool INV>
__device__ __forceinline__ void stage(const cpx<T>* X, cpx<T>* Y, int LS, int P, int W, int lw, int Ns,
                                      const cpx<T>* __restrict__ tw, int tid, int nthr) {
  const int nbf = P / R;
  const int total = nbf * W;
  const int tstride = (2 * P) / (Ns * R);
  for (int idx = tid; idx < total; idx += nthr) {
    const int lane = idx & (W - 1);
    const int j = idx >> lw;
    const int k = j % Ns;
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = X[(j + r * nbf) * LS + lane];
    if (Ns > 1) {
      const int step = tstride * k;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const cpx<T> w = ldg_c<T>(&tw[r * step]);
        v[r] = INV ? cmulc<T>(v[r], w) : cmul<T>(v[r], w);
      }
    }
    dftR<T, R, INV>(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) Y[(base + r * Ns) * LS + lane] = v[r];
  }
}

// Radix plan: up to 8 stages, radices in {16, 8, 4, 2, 3}, one radix per
// 4-bit nibble of `code` (stage s: (code >> 4s) & 15, where 0 stands for 16),
// so that the plan is read without indexing an array of the kernel parameters.
struct RadixPlan {
  int n;
  unsigned code;
};

// Transform the tile held in A (B is scratch of the same size); returns the
// buffer that holds the result.  Ends with a block barrier.
template <typename T, bool INV>
__device__ __forceinline__ cpx<T>* fft_tile(cpx<T>* A, cpx<T>* B, int LS, int P, int W, int lw, const RadixPlan& plan,
                                            const cpx<T>* __restrict__ tw, int tid, int nthr) {
  int Ns = 1;
  cpx<T>* X = A;
  cpx<T>* Y = B;
  for (int s = 0; s < plan.n; ++s) {
    const int nib = (int)((plan.code >> (4 * s)) & 15u);
    switch (nib) {
      case 0: stage<T, 16, INV>(X, Y, LS, P, W, lw, Ns, tw, tid, nthr); Ns *= 16; break;
      case 8: stage<T, 8, INV>(X, Y, LS, P, W, lw, Ns, tw, tid, nthr); Ns *= 8; break;
      case 4: stage<T, 4, INV>(X, Y, LS, P, W, lw, Ns, tw, tid, nthr); Ns *= 4; break;
      case 3: stage<T, 3, INV>(X, Y, LS, P, W, lw, Ns, tw, tid, nthr); Ns *= 3; break;
      default: stage<T, 2, INV>(X, Y, LS, P, W, lw, Ns, tw, tid, nthr); Ns *= 2; break;
    }
    __syncthreads();
    cpx<T>* t = X;
    X = Y;
    Y = t;
  }
  return X;
}

// ---------------------------------------------------------------------------
// Short transforms of the runtime engine (P = 2^a, 4 <= P <= 32): a column is
// held by P lanes of one warp, lane l keeping element l in a register.
// Radix-2 decimation in frequency across the lanes: each stage swaps values
// with lane l ^ h by a warp shuffle, so the stages need neither shared memory
// nor a block barrier.  Both lanes of a pair run the same instructions (no
// divergence): the upper lane negates its own value before the sum and
// multiplies by its twiddle, the lower one by 1.  Lane l ends with mode
// bitrev(l), which the caller writes back to the tile in natural order or
// stores from the register.  Block sizes are whole warps.  The stage engine
// would give such a column to one or two threads (one or two radix-16
// butterflies) while the rest of the block waits; on GB300's FP64 units that
// serial butterfly sets the pass time.  (Longer columns keep the stage
// engine: its radix-16 butterflies take fewer operations per point than
// radix-2 stages.)
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T shfl_xor_t(T v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
template <> __device__ __forceinline__ dfloat shfl_xor_t<dfloat>(dfloat v, int m) {
  return dfloat(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}
template <typename T> __device__ __forceinline__ cpx<T> shfl_xor_c(cpx<T> v, int m) {
  return mk<T>(shfl_xor_t<T>(v.x, m), shfl_xor_t<T>(v.y, m));
}
template <typename T> __device__ __forceinline__ T shfl_idx_t(T v, int src) { return __shfl_sync(0xffffffffu, v, src); }
template <> __device__ __forceinline__ dfloat shfl_idx_t<dfloat>(dfloat v, int src) {
  return dfloat(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
}
template <typename T> __device__ __forceinline__ cpx<T> shfl_idx_c(cpx<T> v, int src) {
  return mk<T>(shfl_idx_t<T>(v.x, src), shfl_idx_t<T>(v.y, src));
}

// Transform the tile's columns with the warp engine; out(c, k, v, ok) receives mode k of column c from
// the lane that holds it (after every lane of the warp has read its element of the tile).  Every
// lane of the warp calls it, so it may exchange values between lanes; ok is false on lanes past the
// tile's last column, whose v is not a mode.
template <typename T, bool INV, typename Out>
__device__ __forceinline__ void fft_cols_warp(const cpx<T>* S, int LS, int P, int W, const cpx<T>* __restrict__ tw,
                                              int tid, int nthr, Out out) {
  const int lane = tid & 31, l = lane & (P - 1);
  const int cpw = 32 / P;                    // columns per warp
  const int lgP = 31 - __clz(P);
  const int kb = (int)(__brev((unsigned)l) >> (32 - lgP));
  const cpx<T> one = mk<T>((T)1, (T)0);
  // warp-uniform loop: every lane of a warp takes part in its shuffles
  for (int c0 = (tid >> 5) * cpw; c0 < W; c0 += (nthr >> 5) * cpw) {
    const int c = c0 + lane / P;
    const bool ok = c < W;
    cpx<T> x = ok ? S[l * LS + c] : mk<T>((T)0, (T)0);
    // span h: lower lane a + b, upper lane (a - b) W_{2h}^{l mod h}, W_{2h}^m = tw[m P / h]
    for (int h = P >> 1; h >= 1; h >>= 1) {
      const bool upper = (l & h) != 0;
      const cpx<T> o = shfl_xor_c<T>(x, h);
      const cpx<T> y = cadd<T>(upper ? mk<T>(-x.x, -x.y) : x, o);
      if (h > 1) {
        const cpx<T> w = upper ? ldg_c<T>(&tw[(l & (h - 1)) * (P / h)]) : one;
        x = INV ? cmulc<T>(y, w) : cmul<T>(y, w);
      } else {
        x = y;
      }
    }
    __syncwarp();  // every lane of the warp has read its element before any is overwritten
    out(c, kb, x, ok);
  }
}

// Transform the tile in place with the warp engine.  Ends with a block barrier.
template <typename T, bool INV>
__device__ __forceinline__ void fft_tile_warp(cpx<T>* S, int LS, int P, int W, const cpx<T>* __restrict__ tw, int tid,
                                              int nthr) {
  fft_cols_warp<T, INV>(S, LS, P, W, tw, tid, nthr, [&](int c, int k, const cpx<T>& v, bool ok) {
    if (ok) S[k * LS + c] = v;
  });
  __syncthreads();
}

// Convolution of a column with the warp engine: forward transform (decimation in frequency,
// natural order in, lane l ends with mode bitrev(l)), times gain(c, k) in registers, inverse
// transform (decimation in time, bit-reversed order in, natural order out) -- no shared-memory round
// trip and no block barrier between the two transforms.  out(c, i, v) receives position i of column
// c from lane i.  DIT stage of span h: the upper lane multiplies its value by W_{2h}^{l mod h} (the
// lower by 1), then lower a + w b, upper a - w b.
template <typename T, typename Gain, typename Out>
__device__ __forceinline__ void conv_cols_warp(const cpx<T>* S, int LS, int P, int W, const cpx<T>* __restrict__ tw,
                                               int tid, int nthr, Gain gain, Out out) {
  const int lane = tid & 31, l = lane & (P - 1);
  const int cpw = 32 / P;
  const int lgP = 31 - __clz(P);
  const cpx<T> one = mk<T>((T)1, (T)0);
  const int kb = (int)(__brev((unsigned)l) >> (32 - lgP));
  for (int c0 = (tid >> 5) * cpw; c0 < W; c0 += (nthr >> 5) * cpw) {
    const int c = c0 + lane / P;
    const bool ok = c < W;
    cpx<T> x = ok ? S[l * LS + c] : mk<T>((T)0, (T)0);
    for (int h = P >> 1; h >= 1; h >>= 1) {
      const bool upper = (l & h) != 0;
      const cpx<T> o = shfl_xor_c<T>(x, h);
      const cpx<T> y = cadd<T>(upper ? mk<T>(-x.x, -x.y) : x, o);
      if (h > 1) {
        const cpx<T> w = upper ? ldg_c<T>(&tw[(l & (h - 1)) * (P / h)]) : one;
        x = cmul<T>(y, w);
      } else {
        x = y;
      }
    }
    if (ok) x = cscale<T>(x, gain(c, kb));
    for (int h = 1; h < P; h <<= 1) {
      const bool upper = (l & h) != 0;
      const cpx<T> t = (h > 1 && upper) ? cmulc<T>(x, ldg_c<T>(&tw[(l & (h - 1)) * (P / h)])) : x;
      const cpx<T> o = shfl_xor_c<T>(t, h);
      x = upper ? csub<T>(o, t) : cadd<T>(t, o);
    }
    if (ok) out(c, l, x);
  }
}

// the warp engine serves the runtime engine's transforms of these lengths
__host__ __device__ constexpr bool warp_fft_len(int P) { return P >= 4 && P <= 32 && (P & (P - 1)) == 0; }

// ---------------------------------------------------------------------------
// Compile-time tile engine for P = 2^a: every stage's radix, stride and
// twiddle step, the tile width W and the block size NT = P W / 16 are known
// at compile time, so the index arithmetic folds to shifts and masks.  The
// tile is transformed in place in one buffer: every thread reads its 16
// elements of a stage into registers, the block synchronises, and the thread
// writes them back (16 = the elements of one radix-16 butterfly, of two
// radix-8 or four radix-4 butterflies).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ct_radix(int rem) {
  // remaining length rem = 2^a: 16s first, a remainder of 32 as 8 x 4, then 8, 4, 2
  return rem == 32 ? 8 : (rem >= 16 ? 16 : rem);
}

// Shared-memory layout of the compile-time engine's tile: element (row i, lane l) of W lanes, rows
// padded to W + 1 elements so that the transposing row-mode accesses (32 consecutive rows of one
// lane) hit distinct banks.  (An XOR swizzle of the 4-lane FP32 tiles removes the stages' bank
// conflicts -- 3.8 wavefronts per access to the minimum 2 -- but its index arithmetic made the
// integer pipe the bottleneck of the x passes: forward 0.643 -> 0.713 ms at 512^3; not used.)
template <typename T, int W> struct CtTile {
  __host__ __device__ static constexpr int at(int i, int l) { return i * (W + 1) + l; }
};

// ZIN: the stage's inputs with r >= R/2 are zero (first stage of a transform
// whose second half is zero padding); ZOUT: its outputs with r >= R/2 are not
// needed (last stage of a transform truncated to its first half).  Both are
// compile-time, so the loads, stores and dead butterfly arithmetic vanish.
template <typename T, int P, int W, int NT, int R, int Ns, bool INV, bool ZIN = false, bool ZOUT = false>
__device__ __forceinline__ void ct_stage(cpx<T>* S, const cpx<T>* __restrict__ tw, int tid) {
  using TL = CtTile<T, W>;
  constexpr int nbf = P / R;
  constexpr int NB = (nbf * W) / NT;
  static_assert((nbf * W) % NT == 0, "tile and block do not match");
  constexpr int tstep = (2 * P) / (Ns * R);
  cpx<T> v[NB][R];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int idx = tid + b * NT;
    const int lane = idx % W, j = idx / W, k = j % Ns;
#pragma unroll
    for (int r = 0; r < R; ++r) v[b][r] = (ZIN && r >= R / 2) ? mk<T>((T)0, (T)0) : S[TL::at(j + r * nbf, lane)];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const cpx<T> w = ldg_c<T>(&tw[r * k * tstep]);
        v[b][r] = INV ? cmulc<T>(v[b][r], w) : cmul<T>(v[b][r], w);
      }
    }
    dftR<T, R, INV>(v[b]);
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int idx = tid + b * NT;
    const int lane = idx % W, j = idx / W, k = j % Ns;
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < (ZOUT ? R / 2 : R); ++r) S[TL::at(base + r * Ns, lane)] = v[b][r];
  }
  __syncthreads();
}

template <typename T, int P, int W, int NT, int Ns, bool INV, bool ZIN, bool ZOUT>
__device__ __forceinline__ void ct_stages(cpx<T>* S, const cpx<T>* __restrict__ tw, int tid) {
  if constexpr (Ns < P) {
    constexpr int R = ct_radix(P / Ns);
    ct_stage<T, P, W, NT, R, Ns, INV, ZIN && Ns == 1, ZOUT && Ns * R == P>(S, tw, tid);
    ct_stages<T, P, W, NT, Ns * R, INV, ZIN, ZOUT>(S, tw, tid);
  }
}

// Stage s of the compile-time plan (forward order): number of stages, radix, Ns.
__host__ __device__ constexpr int ct_nstages(int P) {
  int n = 0, ns = 1;
  while (ns < P) { ns *= ct_radix(P / ns); ++n; }
  return n;
}
__host__ __device__ constexpr int ct_ns(int P, int s) {
  int ns = 1;
  for (int i = 0; i < s; ++i) ns *= ct_radix(P / ns);
  return ns;
}
__host__ __device__ constexpr int ct_rad(int P, int s) { return ct_radix(P / ct_ns(P, s)); }
// the same plan run in reverse radix order (inverse transform of the fused pass)
__host__ __device__ constexpr int ct_rad_rev(int P, int s) { return ct_rad(P, ct_nstages(P) - 1 - s); }
__host__ __device__ constexpr int ct_ns_rev(int P, int s) {
  int ns = 1;
  for (int i = 0; i < s; ++i) ns *= ct_rad_rev(P, i);
  return ns;
}

// Plans of the column kernels, parameterised by the elements a thread holds in a stage: EPT = 16
// is the plan above; EPT = 32 takes radix-32 stages (1024 = 32 x 32, 512 = 32 x 16, 2048 =
// 32 x 8 x 8), one twiddled stage fewer per transform and half the threads per tile.
__host__ __device__ constexpr int ct_radix_e(int rem, int ept) {
  return ept == 32 ? (rem == 64 ? 8 : (rem >= 32 ? 32 : rem)) : ct_radix(rem);
}
__host__ __device__ constexpr int ct_nstages_e(int P, int ept) {
  int n = 0, ns = 1;
  while (ns < P) { ns *= ct_radix_e(P / ns, ept); ++n; }
  return n;
}
__host__ __device__ constexpr int ct_ns_e(int P, int s, int ept) {
  int ns = 1;
  for (int i = 0; i < s; ++i) ns *= ct_radix_e(P / ns, ept);
  return ns;
}
__host__ __device__ constexpr int ct_rad_e(int P, int s, int ept) { return ct_radix_e(P / ct_ns_e(P, s, ept), ept); }
__host__ __device__ constexpr int ct_rad_rev_e(int P, int s, int ept) {
  return ct_rad_e(P, ct_nstages_e(P, ept) - 1 - s, ept);
}
__host__ __device__ constexpr int ct_ns_rev_e(int P, int s, int ept) {
  int ns = 1;
  for (int i = 0; i < s; ++i) ns *= ct_rad_rev_e(P, i, ept);
  return ns;
}

// In-place transform of the tile in S (layout CtTile<T, W>); ends with a barrier.
template <typename T, int P, int W, bool INV, bool ZIN = false, bool ZOUT = false>
__device__ __forceinline__ void fft_tile_ct(cpx<T>* S, const cpx<T>* __restrict__ tw, int tid) {
  ct_stages<T, P, W, P * W / 16, 1, INV, ZIN, ZOUT>(S, tw, tid);
}

}  // namespace flups
