// Device helpers shared by the pass kernels (passes.cu) and the Biot-Savart
// fused kernels (curl.cu): extension geometry, tile loads and stores.
#pragma once
#include <type_traits>
#include "passes.cuh"

namespace flups {

// Real loads/stores of the pass arrays; on the double-float path the caller's
// arrays are FP64 (same element size) and convert on the way in and out.
template <typename T> __device__ __forceinline__ T ld_real(const T* a, long long off, int f64) { return a[off]; }
template <> __device__ __forceinline__ dfloat ld_real<dfloat>(const dfloat* a, long long off, int f64) {
  if (f64) return df_from_double(reinterpret_cast<const double*>(a)[off]);
  const float2 q = reinterpret_cast<const float2*>(a)[off];
  return dfloat(q.x, q.y);
}
template <typename T> __device__ __forceinline__ void st_real(T* a, long long off, T v, int f64) { a[off] = v; }
template <> __device__ __forceinline__ void st_real<dfloat>(dfloat* a, long long off, dfloat v, int f64) {
  if (f64) reinterpret_cast<double*>(a)[off] = df_to_double(v);
  else reinterpret_cast<float2*>(a)[off] = make_float2(v.hi, v.lo);
}

// Index of element (row i, lane l) of a tile: the compile-time engine's layout (WC > 0) or rows of
// LS elements (runtime engine).
// log2 of a power of two, at compile time
__host__ __device__ constexpr int clog2(int x) { return x <= 1 ? 0 : 1 + clog2(x >> 1); }

template <typename T, int WC> __device__ __forceinline__ int tix(int i, int l, int LS) {
  if constexpr (WC > 0) return CtTile<T, WC>::at(i, l);
  else return i * LS + l;
}

// First statement of every pass kernel.  With p.pdl (programmatic dependent launch, sm_90+), the
// kernel was launched before the stream's previous kernel completed: wait until that kernel has
// completed and its writes are visible.  The wait comes before any access to the solve's arrays,
// so read-after-write and write-after-read order between passes is kept; what overlaps is the
// launch and CTA start-up of this pass with the exit of the previous one (the dependent launch
// is triggered as each CTA exits).
__device__ __forceinline__ void pass_entry(const PassParams& p) {
  if (p.pdl) asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Transform type of component `comp` (4 bits per component).
__device__ __forceinline__ int comp_type(const PassParams& p, int comp) { return (p.ctypes >> (4 * comp)) & 15; }


// ---------------------------------------------------------------------------
// Extension geometry (Sections 2.2, 2.3).  Data index i (already mirrored for
// the unbounded-left semi types) -> positions and signs in the extension.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int base_type(int t) {
  return t == T_UE ? T_EU : (t == T_UO ? T_OU : t);
}

__device__ __forceinline__ int images(int t, int center, int N, int i, int* pos, int* sg) {
  int n = 0;
  if (center == C_CELL) {
    switch (t) {
      case T_PER: case T_UNB: pos[0] = i; sg[0] = 1; return 1;
      case T_EE: pos[0] = i; sg[0] = 1; pos[1] = 2 * N - 1 - i; sg[1] = 1; return 2;
      case T_OO: pos[0] = i; sg[0] = 1; pos[1] = 2 * N - 1 - i; sg[1] = -1; return 2;
      case T_EO:
        pos[0] = i; sg[0] = 1; pos[1] = 2 * N - 1 - i; sg[1] = -1;
        pos[2] = 2 * N + i; sg[2] = -1; pos[3] = 4 * N - 1 - i; sg[3] = 1; return 4;
      case T_OE:
        pos[0] = i; sg[0] = 1; pos[1] = 2 * N - 1 - i; sg[1] = 1;
        pos[2] = 2 * N + i; sg[2] = -1; pos[3] = 4 * N - 1 - i; sg[3] = -1; return 4;
      case T_EU: pos[0] = i; sg[0] = 1; pos[1] = 4 * N - 1 - i; sg[1] = 1; return 2;
      case T_OU: pos[0] = i; sg[0] = 1; pos[1] = 4 * N - 1 - i; sg[1] = -1; return 2;
    }
    return 0;
  }
  switch (t) {
    case T_PER: if (i < N) { pos[0] = i; sg[0] = 1; return 1; } return 0;
    case T_UNB: pos[0] = i; sg[0] = 1; return 1;
    case T_EE:
      pos[n] = i; sg[n++] = 1;
      if (i > 0 && i < N) { pos[n] = 2 * N - i; sg[n++] = 1; }
      return n;
    case T_OO:
      if (i > 0 && i < N) { pos[0] = i; sg[0] = 1; pos[1] = 2 * N - i; sg[1] = -1; return 2; }
      return 0;
    case T_OE:
      if (i >= 1) { pos[n] = i; sg[n++] = 1; pos[n] = 2 * N + i; sg[n++] = -1; }
      if (i >= 1 && i <= N - 1) { pos[n] = 2 * N - i; sg[n++] = 1; pos[n] = 4 * N - i; sg[n++] = -1; }
      return n;
    case T_EO:
      if (i <= N - 1) { pos[n] = i; sg[n++] = 1; pos[n] = 2 * N - i; sg[n++] = -1; }
      if (i >= 1 && i <= N - 1) { pos[n] = 2 * N + i; sg[n++] = -1; pos[n] = 4 * N - i; sg[n++] = 1; }
      return n;
    case T_EU:
      pos[n] = i; sg[n++] = 1;
      if (i >= 1) { pos[n] = 4 * N - i; sg[n++] = 1; }
      return n;
    case T_OU:
      if (i >= 1) { pos[0] = i; sg[0] = 1; pos[1] = 4 * N - i; sg[1] = -1; return 2; }
      return 0;
  }
  return 0;
}

// Positions of the extension that hold zeros (padding, odd faces); up to 3 ranges.
__device__ __forceinline__ int zero_ranges(int t, int center, int N, int* lo, int* hi) {
  if (center == C_CELL) {
    if (t == T_UNB) { lo[0] = N; hi[0] = 2 * N; return 1; }
    if (t == T_EU || t == T_OU) { lo[0] = N; hi[0] = 3 * N; return 1; }
    return 0;
  }
  switch (t) {
    case T_UNB: lo[0] = N + 1; hi[0] = 2 * N; return 1;
    case T_OO: lo[0] = 0; hi[0] = 1; lo[1] = N; hi[1] = N + 1; return 2;
    case T_OE: lo[0] = 0; hi[0] = 1; lo[1] = 2 * N; hi[1] = 2 * N + 1; return 2;
    case T_EO: lo[0] = N; hi[0] = N + 1; lo[1] = 3 * N; hi[1] = 3 * N + 1; return 2;
    case T_EU: lo[0] = N + 1; hi[0] = 3 * N; return 1;
    case T_OU: lo[0] = 0; hi[0] = 1; lo[1] = N + 1; hi[1] = 3 * N; return 2;
  }
  return 0;
}

// Extension position holding data index i on output, or -1 when the value is
// forced to 0 (odd node face).  Node periodic phi_N := phi_0 (Section 2.1).
__device__ __forceinline__ int primary_pos(int t, int center, int N, int i) {
  if (center == C_NODE) {
    if (t == T_PER && i == N) return 0;
    if ((t == T_OO) && (i == 0 || i == N)) return -1;
    if ((t == T_OE || t == T_OU) && i == 0) return -1;
    if (t == T_EO && i == N) return -1;
  }
  return i;
}

// ---------------------------------------------------------------------------
// Shared helpers.
// ---------------------------------------------------------------------------
template <typename T, int WC = 0>
__device__ __forceinline__ void zero_fill(cpx<T>* S, int LS, int W, int lo, int hi, int tid, int nthr) {
  // W is a power of two (index arithmetic by shifts: W is a runtime value in the runtime engine)
  const int tot = (hi - lo) * W, lw = 31 - __clz(W);
  for (int idx = tid; idx < tot; idx += nthr) {
    const int lane = idx & (W - 1);
    const int j = lo + (idx >> lw);
    S[tix<T, WC>(j, lane, LS)] = mk<T>((T)0, (T)0);
  }
}

// Build the two-pencil extension of real data (pencils q0 + c, c < 2W).
// skip_zero: the first FFT stage never reads the zero-padding rows (half-zero input)
template <typename T, int WC = 0>
__device__ __forceinline__ void load_real_ext(const PassParams& p, int type, const T* __restrict__ in, cpx<T>* S,
                                              int q0, int tid, int nthr, bool skip_zero = false) {
  const int W = WC ? WC : p.W, LS = WC ? WC + 1 : p.LS, N = p.N, nd = p.n_data, lw = WC ? clog2(WC) : p.lw;
  const int t = base_type(type);
  const bool rev = is_reversed(type);
  int lo[3], hi[3];
  const int nz = skip_zero ? 0 : zero_ranges(t, p.center, N, lo, hi);
  for (int r = 0; r < nz; ++r) zero_fill<T, WC>(S, LS, W, lo[r], hi[r], tid, nthr);
  T* Sr = reinterpret_cast<T*>(S);
  const int W2 = 2 * W;
  const bool rowmode = p.axis == 0;
  const int lgM = 31 - __clz(nd), M = 1 << lgM, rem = nd - M;
  if (WC > 0 && rowmode) {
    // compile-time tile in row mode: a thread takes position i of both pencils of a lane (two
    // coalesced loads, rows q0 + 2 lane and q0 + 2 lane + 1) and writes each image as one complex
    // (a, b) -- one 8-byte shared store instead of two 4-byte ones.  Index space: rows of
    // M = 2^floor(log2 nd) values, then the nd - M remaining ones.
    const int tot_main = W << lgM, tot = tot_main + W * rem;
    constexpr int LB = std::is_same<T, dfloat>::value ? 1 : 4;
    for (int base = tid; base < tot; base += LB * nthr) {
      T va[LB], vb[LB];
      int ll[LB], ii[LB];
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        const int idx = base + u * nthr;
        int lane = 0, i = -1;
        if (idx < tot) {
          if (idx < tot_main) { i = idx & (M - 1); lane = idx >> lgM; }
          else { const int r = idx - tot_main; lane = r / rem; i = M + r % rem; }
        }
        ll[u] = lane;
        ii[u] = i;
        const int qa = q0 + 2 * lane;
        const long long off = (long long)qa * p.ai.ls + (long long)i * p.ai.js;
        va[u] = (i >= 0 && qa < p.npen) ? ld_real<T>(in, off, p.in_f64) : (T)0;
        vb[u] = (i >= 0 && qa + 1 < p.npen) ? ld_real<T>(in, off + p.ai.ls, p.in_f64) : (T)0;
      }
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        if (ii[u] < 0) continue;
        const int dix = rev ? nd - 1 - ii[u] : ii[u];
        int pos[4], sg[4];
        const int n = images(t, p.center, N, dix, pos, sg);
        for (int k = 0; k < n; ++k)
          S[tix<T, WC>(pos[k], ll[u], LS)] = sg[k] > 0 ? mk<T>(va[u], vb[u]) : mk<T>(-va[u], -vb[u]);
      }
    }
    return;
  }
  // runtime tiles in row mode: index i fastest over a power-of-two stride (1 << ndlog) >= nd
  const int tot = rowmode ? (W2 << p.ndlog) : nd * W2;
  // batches of LOADB independent loads per thread before their values are used (latency
  // hiding); the double-float path converts FP64 words on load and runs fastest unbatched
  constexpr int LOADB = std::is_same<T, dfloat>::value ? 1 : 8;
  for (int base = tid; base < tot; base += LOADB * nthr) {
    T v[LOADB];
    int cc[LOADB], ii[LOADB];
#pragma unroll
    for (int u = 0; u < LOADB; ++u) {
      const int idx = base + u * nthr;
      int c = 0, i = -1;
      if (idx < tot) {
        if (rowmode) { i = idx & ((1 << p.ndlog) - 1); c = idx >> p.ndlog; if (i >= nd) i = -1; }
        else { c = idx & (W2 - 1); i = idx >> (lw + 1); }
      }
      cc[u] = c;
      ii[u] = i;
      const int q = q0 + c;
      v[u] = (i >= 0 && q < p.npen) ? ld_real<T>(in, (long long)q * p.ai.ls + (long long)i * p.ai.js, p.in_f64) : (T)0;
    }
#pragma unroll
    for (int u = 0; u < LOADB; ++u) {
      if (ii[u] < 0) continue;
      const int dix = rev ? nd - 1 - ii[u] : ii[u];
      int pos[4], sg[4];
      const int n = images(t, p.center, N, dix, pos, sg);
      const int lane = cc[u] >> 1, part = cc[u] & 1;
      for (int k = 0; k < n; ++k) Sr[2 * tix<T, WC>(pos[k], lane, LS) + part] = sg[k] > 0 ? v[u] : -v[u];
    }
  }
}

// Store data values of both pencils of every lane from the inverse-transformed extension.
template <typename T, int WC = 0>
__device__ __forceinline__ void store_real_data(const PassParams& p, int type, T* __restrict__ out, const cpx<T>* S,
                                                int q0, int tid, int nthr) {
  const int W = WC ? WC : p.W, LS = WC ? WC + 1 : p.LS, N = p.N, nd = p.n_data, lw = WC ? clog2(WC) : p.lw;
  const int t = base_type(type);
  const bool rev = is_reversed(type);
  const int W2 = 2 * W;
  const bool rowmode = p.axis == 0;
  const int lgM = 31 - __clz(nd), M = 1 << lgM, rem = nd - M;
  if (WC > 0 && rowmode) {
    // compile-time tile in row mode: a thread reads one complex (a, b) of a lane and writes
    // position i of both pencils (index space as in load_real_ext)
    const int tot_main = W << lgM, tot = tot_main + W * rem;
    for (int idx = tid; idx < tot; idx += nthr) {
      int lane, i;
      if (idx < tot_main) { i = idx & (M - 1); lane = idx >> lgM; }
      else { const int r = idx - tot_main; lane = r / rem; i = M + r % rem; }
      const int qa = q0 + 2 * lane;
      if (qa >= p.npen) continue;
      const int ii = rev ? nd - 1 - i : i;
      const int pos = primary_pos(t, p.center, N, ii);
      cpx<T> z = mk<T>((T)0, (T)0);
      if (pos >= 0) z = S[tix<T, WC>(pos, lane, LS)];
      const long long off = (long long)qa * p.ao.ls + (long long)i * p.ao.js;
      st_real<T>(out, off, z.x, p.out_f64);
      if (qa + 1 < p.npen) st_real<T>(out, off + p.ao.ls, z.y, p.out_f64);
    }
    return;
  }
  const int tot = rowmode ? (W2 << p.ndlog) : nd * W2;
  for (int idx = tid; idx < tot; idx += nthr) {
    int c, i;
    if (rowmode) { i = idx & ((1 << p.ndlog) - 1); c = idx >> p.ndlog; if (i >= nd) continue; }
    else { c = idx & (W2 - 1); i = idx >> (lw + 1); }
    const int q = q0 + c;
    if (q >= p.npen) continue;
    const int ii = rev ? nd - 1 - i : i;
    const int pos = primary_pos(t, p.center, N, ii);
    T v = (T)0;
    if (pos >= 0) {
      const cpx<T> z = S[tix<T, WC>(pos, c >> 1, LS)];
      v = (c & 1) ? z.y : z.x;
    }
    st_real<T>(out, (long long)q * p.ao.ls + (long long)i * p.ao.js, v, p.out_f64);
  }
}

// Spectrum of pencil a (part 0) or b (part 1) at mode k from the packed FFT.
template <typename T>
__device__ __forceinline__ cpx<T> split(cpx<T> zk, cpx<T> zm, int part) {
  const T h = T(0.5);
  return part == 0 ? mk<T>(h * (zk.x + zm.x), h * (zk.y - zm.y)) : mk<T>(h * (zk.y + zm.y), h * (zm.x - zk.x));
}


template <typename T, int WC = 0>
__device__ __forceinline__ void load_cplx(const PassParams& p, const cpx<T>* __restrict__ in, cpx<T>* S, int q0,
                                          int tid, int nthr, bool skip_zero = false) {
  const int W = WC ? WC : p.W, LS = WC ? WC + 1 : p.LS, nu = p.n_use, lw = WC ? clog2(WC) : p.lw;
  if (nu < p.P && !skip_zero) zero_fill<T, WC>(S, LS, W, nu, p.P, tid, nthr);
  const bool rowmode = p.axis == 0;
  const int tot = rowmode ? (W << p.ndlog) : nu * W;
  constexpr int LOADB = 8;
  for (int base = tid; base < tot; base += LOADB * nthr) {
    cpx<T> v[LOADB];
    int ll[LOADB], ii[LOADB];
#pragma unroll
    for (int u = 0; u < LOADB; ++u) {
      const int idx = base + u * nthr;
      int lane = 0, i = -1;
      if (idx < tot) {
        if (rowmode) { i = idx & ((1 << p.ndlog) - 1); lane = idx >> p.ndlog; if (i >= nu) i = -1; }
        else { lane = idx & (W - 1); i = idx >> lw; }
      }
      ll[u] = lane;
      ii[u] = i;
      const int q = q0 + lane;
      v[u] = (i >= 0 && q < p.npen) ? in[(long long)q * p.ai.ls + (long long)i * p.ai.js] : mk<T>((T)0, (T)0);
    }
#pragma unroll
    for (int u = 0; u < LOADB; ++u)
      if (ii[u] >= 0) S[tix<T, WC>(ii[u], ll[u], LS)] = v[u];
  }
}

template <typename T, int WC = 0>
__device__ __forceinline__ void store_cplx_data(const PassParams& p, cpx<T>* __restrict__ out, const cpx<T>* S, int q0,
                                                int tid, int nthr) {
  const int W = WC ? WC : p.W, LS = WC ? WC + 1 : p.LS, nd = p.n_data, lw = WC ? clog2(WC) : p.lw;
  const bool rowmode = p.axis == 0;
  const int tot = rowmode ? (W << p.ndlog) : nd * W;
  for (int idx = tid; idx < tot; idx += nthr) {
    int lane, i;
    if (rowmode) { i = idx & ((1 << p.ndlog) - 1); lane = idx >> p.ndlog; if (i >= nd) continue; }
    else { lane = idx & (W - 1); i = idx >> lw; }
    const int q = q0 + lane;
    if (q >= p.npen) continue;
    const int pos = (p.type == T_PER && p.center == C_NODE && i == p.N) ? 0 : i;
    out[(long long)q * p.ao.ls + (long long)i * p.ao.js] = S[tix<T, WC>(pos, lane, LS)];
  }
}

}  // namespace flups
