// C ABI of the solver (include/flups_gpu.h): planner, device memory, launches.
//
// Planning follows Section 1 and Section "Methodology": each direction is
// classified from its two face conditions into periodic, unbounded, one of
// the four symmetric types of Table 1 or a semi-unbounded type (Section
// 2.3.2); directions run in order of cost (symmetric, semi-unbounded,
// periodic, unbounded); the first periodic/unbounded direction met on real
// data is an R2C transform, later ones are C2C.  The last direction is fused:
// forward transform, multiplication by G^ (eq. poisson), inverse transform.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "flups_gpu.h"
#include "green.cuh"
#include "passes.cuh"

using namespace flups;

namespace {

thread_local std::string g_last_cuda = "no error";

int cuda_fail(cudaError_t e, const char* where) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  g_last_cuda = buf;
  return FLUPS_ECUDA;
}
#define CK(call)                                   \
  do {                                             \
    cudaError_t e__ = (call);                      \
    if (e__ != cudaSuccess) return cuda_fail(e__, #call); \
  } while (0)

bool is_2a3b(long n) {
  if (n < 2) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

RadixPlan radix_plan(int P) {
  RadixPlan rp{};
  int p = P;
  auto push = [&](int r) { rp.code |= (unsigned)r << (4 * rp.n); rp.n++; };
  int a = 0;
  while (p % 2 == 0) { ++a; p /= 2; }
  // 2^a as 16s and one 8 or 4; a remainder of 2^1 is folded into 8 x 4
  int n16 = a / 4, rem = a % 4;
  if (rem == 1 && n16 > 0) { --n16; rem = 5; }
  for (int i = 0; i < n16; ++i) push(0);  // nibble 0 encodes radix 16
  if (rem == 5) { push(8); push(4); }
  else if (rem == 3) push(8);
  else if (rem == 2) push(4);
  else if (rem == 1) push(2);
  while (p % 3 == 0) { push(3); p /= 3; }
  return rp;
}

// Direction type from its two faces (Section 1 categories, Table 1 parities).
int classify(int l, int r, int* type) {
  auto ok = [](int b) { return b == FLUPS_EVEN || b == FLUPS_ODD || b == FLUPS_PER || b == FLUPS_UNB; };
  if (!ok(l) || !ok(r)) return FLUPS_EINVAL;
  if (l == FLUPS_PER || r == FLUPS_PER) {
    if (l != r) return FLUPS_EBC;
    *type = T_PER;
    return FLUPS_OK;
  }
  if (l == FLUPS_UNB && r == FLUPS_UNB) { *type = T_UNB; return FLUPS_OK; }
  if (l == FLUPS_UNB) { *type = (r == FLUPS_EVEN) ? T_UE : T_UO; return FLUPS_OK; }
  if (r == FLUPS_UNB) { *type = (l == FLUPS_EVEN) ? T_EU : T_OU; return FLUPS_OK; }
  if (l == FLUPS_EVEN) *type = (r == FLUPS_EVEN) ? T_EE : T_EO;
  else *type = (r == FLUPS_EVEN) ? T_OE : T_OO;
  return FLUPS_OK;
}

int cost_class(int t) {
  if (t >= T_EE && t <= T_OO) return 1;
  if (t >= T_EU) return 2;
  if (t == T_PER) return 3;
  return 4;
}

bool is_quarter_t(int t) { return t == T_EO || t == T_OE; }
bool is_semi_t(int t) { return t >= T_EU; }
bool is_unb_like(int t) { return t == T_UNB || is_semi_t(t); }

enum Role { R_R2R = 0, R_R2C = 1, R_C2C = 2 };

struct DirPlan {
  int type = 0, n_data = 0, N = 0, P = 0, role = 0, nm = 0, gext = 0, unb = 0;
  double h = 0, L = 0, wscale = 0, wshift = 0;
  RadixPlan rp{};
  void* tw = nullptr;
};

struct Launch {
  int kind;
  PassParams p;
  dim3 grid;
  int nthr;
  size_t smem;
  int user_in, user_out;  // 1: the pointer is the caller's rhs / phi
  int in_buf, out_buf;    // workspace buffer read / written: 1 = W1, 2 = W2, 0 = none
  double bytes, flops;    // algorithmic bytes moved and nominal FFT flops (5 P log2 P per complex FFT)
  int gnthr;              // x passes on the register-chained stages: the generic row kernel's block
  size_t gsmem;           // size and shared memory, used when the pass reads or writes pinned host memory
};

}  // namespace

struct flups_topo_s {
  int n[3];
  int center, ncomp, prec;
};

struct flups_solver_s {
  flups_topo_s topo;
  int bc[3][3][2];
  double h[3], L[3];
  int green, op, diff;
  double eps_over_h, eps;
  int types[3];        // per direction, the (first component's) type that sets the plan's geometry
  int tf[3][3];        // [comp][dir] transform type of the source
  int tu[3][3];        // [comp][dir] transform type of the result (Biot-Savart: the curl's conditions)
  void* dsym[3] = {nullptr, nullptr, nullptr};
  DirPlan dir[3];
  int order[3];
  int dims[3][3];     // array dims after 0, 1, 2 forward passes
  int pitch[3];       // x pitch of those arrays (the workspaces' rows padded to 16 bytes)
  int cplx[3];        // element type of those arrays (0 real, 1 complex)
  size_t elems1 = 0, elems2 = 0;
  void* W1 = nullptr;
  void* W2 = nullptr;
  void* green_dev = nullptr;
  int green_pitch = 0;          // x pitch (elements) of the stored spectrum
  bool share_green = false;     // look the stored spectrum up in (and add it to) the process-wide cache
  std::string green_key;        // its cache key when shared
  void* gmaps_dev = nullptr;    // TMA tensor maps of the stored spectrum (fused column pass)
  int* errflag = nullptr;       // device word set by bounded waits that give up
  int dbg_wait = 0;             // test hook (flups_debug_wait_limit): waits that give up at once
  void* tabs[3] = {nullptr, nullptr, nullptr};
  void* stage = nullptr;  // device copy of the caller's host arrays (flups_solve_host)
  size_t user_bytes = 0;
  double green_bytes = 0, model_bytes = 0;
  size_t ws_bytes = 0;
  std::vector<Launch> passes;
  bool ready = false;
  bool shared = false;    // set up without its own workspace (solves pass one in)
  size_t ws_need = 0;     // bytes of workspace one solve needs (W1 + W2, 256-aligned, + the status block)
};

namespace {

size_t esize(int prec) { return prec == FLUPS_F32 ? 4 : 8; }

// Twiddles exp(-2 pi i m/(2P)), m = 0..2P-1, in extended precision then rounded once.
static int make_twiddles_uncached(int P, int prec, void** out) {
  const int M = 2 * P;
  std::vector<double> re(M), im(M);
  for (int m = 0; m < M; ++m) {
    const long double a = 3.141592653589793238462643383279502884L * (long double)m / (long double)P;
    re[m] = (double)cosl(a);
    im[m] = (double)(-sinl(a));
  }
  const size_t bytes = (size_t)M * 2 * esize(prec);
  void* d = nullptr;
  if (prec != FLUPS_F64E) CK(cudaMalloc(&d, bytes));
  if (prec == FLUPS_F32) {
    std::vector<float> h(2 * M);
    for (int m = 0; m < M; ++m) { h[2 * m] = (float)re[m]; h[2 * m + 1] = (float)im[m]; }
    CK(cudaMemcpy(d, h.data(), bytes, cudaMemcpyHostToDevice));
  } else if (prec == FLUPS_F64E) {
    // double-float pairs (hi, lo) of the re and im parts, from the extended-precision values
    std::vector<float> h(4 * M);
    for (int m = 0; m < M; ++m) {
      const long double a = 3.141592653589793238462643383279502884L * (long double)m / (long double)P;
      const long double c = cosl(a), sn = -sinl(a);
      const float ch = (float)c, sh = (float)sn;
      h[4 * m] = ch;
      h[4 * m + 1] = (float)(c - (long double)ch);
      h[4 * m + 2] = sh;
      h[4 * m + 3] = (float)(sn - (long double)sh);
    }
    CK(cudaMalloc(&d, (size_t)M * 16));
    CK(cudaMemcpy(d, h.data(), (size_t)M * 16, cudaMemcpyHostToDevice));
    *out = d;
    return FLUPS_OK;
  } else {
    std::vector<double> h(2 * M);
    for (int m = 0; m < M; ++m) { h[2 * m] = re[m]; h[2 * m + 1] = im[m]; }
    CK(cudaMemcpy(d, h.data(), bytes, cudaMemcpyHostToDevice));
  }
  *out = d;
  return FLUPS_OK;
}

// Twiddle tables are shared by every plan of a process: one table per (device,
// P, precision), created on first use and kept until exit (a few KB each), so
// that plan setup and teardown allocate and free no twiddles.
std::mutex g_tw_mu;
std::map<long long, void*> g_tw_cache;

int make_twiddles(int P, int prec, void** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  const long long key = ((long long)dev << 40) | ((long long)prec << 32) | (long long)P;
  std::lock_guard<std::mutex> lk(g_tw_mu);
  auto it = g_tw_cache.find(key);
  if (it != g_tw_cache.end()) {
    *out = it->second;
    return FLUPS_OK;
  }
  void* d = nullptr;
  const int rc = make_twiddles_uncached(P, prec, &d);
  if (rc) return rc;
  g_tw_cache[key] = d;
  *out = d;
  return FLUPS_OK;
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5));
    double pp = 0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        const double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      const double z1 = z;
      z = z1 - p1 / pp;
      if (std::fabs(z - z1) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}


// Strides of an array of d[0] x d[1] x d[2] values (x fastest) whose x rows are `pitch` apart.
ArrDesc arr_desc(const int* d, int pitch, int axis) {
  ArrDesc a{};
  const long long tot = (long long)pitch * d[1] * d[2];
  a.cs = tot;
  if (axis == 0) { a.ls = pitch; a.js = 1; a.os = 0; }
  else if (axis == 1) { a.ls = 1; a.js = pitch; a.os = (long long)pitch * d[1]; }
  else { a.ls = 1; a.js = (long long)pitch * d[1]; a.os = pitch; }
  return a;
}

int ilog2(int w) { int l = 0; while ((1 << l) < w) ++l; return l; }

int pack3(int a, int b, int c) { return a | (b << 4) | (c << 8); }
size_t esz(int prec) { return prec == FLUPS_F32 ? 4 : 8; }

// Geometry family of a direction type: the components of a vector field must
// share it per direction (same extension length and mode layout).
int family(int t) {
  switch (t) {
    case T_PER: return 0;
    case T_UNB: return 1;
    case T_EE: case T_OO: return 2;
    case T_EO: case T_OE: return 3;
    case T_EU: case T_OU: return 4;
    default: return 5;
  }
}

int swap_parity(int b) { return b == FLUPS_EVEN ? FLUPS_ODD : (b == FLUPS_ODD ? FLUPS_EVEN : b); }

// Derivative symbol per extension mode kk of a P-periodic direction: the
// signed wavenumber w = 2 pi s/(P h), s = kk or kk - P, zero at the Nyquist
// mode, or the finite-difference symbols (Section "Application: the
// Biot-Savart solver"): order 2 sin(wh)/h, order 4 (4/3 sin wh - 1/6 sin 2wh)/h,
// order 6 (3/2 sin wh - 3/10 sin 2wh + 1/30 sin 3wh)/h.
int make_dsym(int P, double h, int diff, int prec, void** out, cudaStream_t st) {
  std::vector<double> v(P);
  for (int kk = 0; kk < P; ++kk) {
    const int sgn = (2 * kk <= P) ? kk : kk - P;
    const double w = 2.0 * M_PI * sgn / (P * h);
    double sym;
    if (2 * kk == P) sym = 0.0;
    else if (diff == FLUPS_DIFF_FD2) sym = std::sin(w * h) / h;
    else if (diff == FLUPS_DIFF_FD4) sym = (4.0 / 3.0 * std::sin(w * h) - std::sin(2 * w * h) / 6.0) / h;
    else if (diff == FLUPS_DIFF_FD6)
      sym = (1.5 * std::sin(w * h) - 0.3 * std::sin(2 * w * h) + std::sin(3 * w * h) / 30.0) / h;
    else sym = w;
    v[kk] = sym;
  }
  const size_t bytes = (size_t)P * esz(prec);
  CK(cudaMallocAsync(out, bytes, st));
  if (prec == FLUPS_F32) {
    std::vector<float> f(v.begin(), v.end());
    CK(cudaMemcpyAsync(*out, f.data(), bytes, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  } else if (prec == FLUPS_F64E) {
    // double-float pairs (hi = nearest float, lo = nearest float of the remainder)
    std::vector<float> f(2 * (size_t)P);
    for (int kk = 0; kk < P; ++kk) {
      f[2 * kk] = (float)v[kk];
      f[2 * kk + 1] = (float)(v[kk] - (double)f[2 * kk]);
    }
    CK(cudaMemcpyAsync(*out, f.data(), bytes, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  } else {
    CK(cudaMemcpyAsync(*out, v.data(), bytes, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  }
  return FLUPS_OK;
}

// Tile shape: W lanes (power of 2) per CTA within a 2 x 32 KB ping-pong
// shared-memory budget; about one radix-16 butterfly per thread and stage.
void tile_shape(int P, int prec, int npen, bool packed, int* W, int* nthr, int share = 1) {
  const int budget = (prec == FLUPS_F32 ? 4096 : 2048) / share;  // complex elements per buffer
  int w = 1;
  while (w * 2 * P <= budget && w < 64) w *= 2;
  int need = packed ? (npen + 1) / 2 : npen;
  int cap = 1;
  while (cap < need) cap *= 2;
  if (w > cap) w = cap;
  if (w < 1) w = 1;
  *W = w;
  const int tmax = prec == FLUPS_F32 ? 512 : 256;
  int t = (P * w + 15) / 16;
  t = ((t + 31) / 32) * 32;
  if (t < 64) t = 64;
  if (t > tmax) t = tmax;
  *nthr = t;
}

void fill_geom(Launch& L, const DirPlan& dp, int axis, const int* din, const int* dout, int prec, bool packed,
               int center, int ncomp, int share = 1, int pin = -1, int pout = -1) {
  PassParams& p = L.p;
  p.ai = arr_desc(din, pin < 0 ? din[0] : pin, axis);
  p.ao = arr_desc(dout, pout < 0 ? dout[0] : pout, axis);
  p.axis = axis;
  p.npen = axis == 0 ? din[1] * din[2] : din[0];
  int W, nthr;
  int wct = share == 1 ? ct_tile_width(dp.P, prec, axis, L.kind) : 0;  // the curl pass keeps the runtime engine
  const int other = axis == 0 ? 1 : (axis == 1 ? din[2] : din[1]);
  auto ctas = [&](int w) { return (long long)((p.npen + (packed ? 2 * w : w) - 1) / (packed ? 2 * w : w)) * other * ncomp; };
  // small grid: narrow compile-time tiles where they are built (FP32, P = 64), else narrower runtime
  // tiles -- more CTAs either way
  if (wct && ctas(wct) < 2 * 152) wct = ct_small_width(dp.P, prec);
  if (wct) {
    W = wct;
    nthr = dp.P * W / 16;
    p.ct = 1;
    p.LS = W + 1;
  } else {
    tile_shape(dp.P, prec, p.npen, packed, &W, &nthr, share);
    while (W > 1 && ctas(W) < 2 * 152) W /= 2;
    {
      // stage engine: 16 elements per thread; warp engine (P <= 32): a column on P lanes
      const bool wfft = warp_fft_len(dp.P);
      int t = wfft ? W * dp.P : (dp.P * W + 15) / 16;
      t = ((t + 31) / 32) * 32;
      nthr = std::min(std::max(t, wfft ? 32 : 64), prec == FLUPS_F32 ? 512 : 256);
    }
    p.ct = 0;
    p.LS = (axis == 0 && W >= 8) ? W + 1 : W;
  }
  p.W = W;
  p.lw = ilog2(W);
  p.type = dp.type;
  p.ctypes = dp.type | (dp.type << 4) | (dp.type << 8);
  p.center = center;
  p.N = dp.N;
  p.n_data = dp.n_data;
  p.P = dp.P;
  p.n_modes = dp.nm;
  p.n_use = (dp.type == T_PER) ? dp.N : dp.n_data;
  p.hz = (p.ct && dp.type == T_UNB && center == FLUPS_CELL && 2 * dp.n_data == dp.P) ? 1 : 0;
  {
    int m = std::max(std::max(p.n_data, p.n_use), p.n_modes);
    p.ndlog = ilog2(m);
    p.hlog = ilog2(dp.P / 2 + 1);
  }
  p.plan = dp.rp;
  p.tw = dp.tw;
  const int per_tile = packed ? 2 * W : W;
  L.grid = dim3((p.npen + per_tile - 1) / per_tile, axis == 0 ? 1 : (axis == 1 ? din[2] : din[1]), ncomp);
  L.nthr = nthr;
  L.smem = (p.ct ? 1 : 2) * (size_t)dp.P * p.LS * 2 * esize(prec) + 16 * 2 * W + 16;
  p.ept = 16;
  if (p.ct && axis != 0 && (L.kind == K_FWD_C2C || L.kind == K_INV_C2C || L.kind == K_FUSED_C2C)) {
    // column kernels: 128-byte alignment of the tile and a 128-byte block for their mbarriers;
    // EPT elements per thread and stage
    L.smem += 256;
    p.ept = ct_col_ept(dp.P, prec, L.kind);
    L.nthr = dp.P * W / p.ept;
  }
}

// CTAs per SM the compile-time kernels are built for (their __launch_bounds__ minimum).
int ct_min_blocks(const PassParams& p, int nthr, int prec) {
  nthr = std::max(nthr, 32);  // a CTA narrower than a warp holds a whole warp
  if (p.ept == 32) return std::max(1, 512 / nthr);
  return std::max(1, (prec == FLUPS_F32 ? 1024 : 512) / nthr);
}

// Sampling parameters of the stored spectrum (every direction's Green index extent, the
// unbounded-like directions sampled in real space, the spectral ones by wavenumber).
GreenSampleParams green_params(const flups_solver_s* s) {
  GreenSampleParams q{};
  int du = 0;
  for (int d = 0; d < 3; ++d) {
    const DirPlan& dp = s->dir[d];
    q.gext[d] = dp.gext;
    q.unb[d] = dp.unb;
    q.h[d] = dp.h;
    q.wscale[d] = dp.wscale;
    q.wshift[d] = dp.wshift;
    du += dp.unb;
  }
  q.du = du;
  q.kernel = s->green == FLUPS_HEJ0 ? 1 : 0;
  q.hej_m = (s->green >= FLUPS_HEJ2 && s->green <= FLUPS_HEJ10) ? s->green / 2 : 1;
  q.eps = s->eps;
  q.hmax = std::fmax(s->h[0], std::fmax(s->h[1], s->h[2]));
  gauss_legendre(GL_N, q.gl_x, q.gl_w);
  return q;
}

// FP64 samples G(k_s, r_u) of the stored spectrum's kernel, x fastest over the Green extents.
cudaError_t sample_green(const flups_solver_s* s, const GreenSampleParams& q, double* g64, cudaStream_t st) {
  return (s->green == FLUPS_LGF2) ? launch_lgf(g64, q.gext, q.h, st) : launch_green_sample(g64, q, st);
}

int setup_green_compute(flups_solver_s* s, cudaStream_t st) {
  const int prec = s->topo.prec;
  int du = 0;
  for (int d = 0; d < 3; ++d) du += s->dir[d].unb;
  double Pprod = 1.0;
  for (int d = 0; d < 3; ++d) Pprod *= s->dir[d].P;
  if (du == 0) {
    // closed form on the fly: per-direction |w|^2 (or the 7-point FD symbol for LGF2)
    for (int d = 0; d < 3; ++d) {
      const DirPlan& dp = s->dir[d];
      std::vector<double> tab(dp.gext);
      for (int g = 0; g < dp.gext; ++g) {
        const double w = dp.wscale * (g + dp.wshift);
        if (s->green == FLUPS_LGF2) {
          const double sn = std::sin(0.5 * w * dp.h);
          tab[g] = 4.0 * sn * sn / (dp.h * dp.h);
        } else {
          tab[g] = w * w;
        }
      }
      const size_t bytes = dp.gext * esize(prec);
      CK(cudaMallocAsync(&s->tabs[d], bytes, st));
      if (prec == FLUPS_F32) {
        std::vector<float> f(tab.begin(), tab.end());
        CK(cudaMemcpyAsync(s->tabs[d], f.data(), bytes, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
      } else {
        CK(cudaMemcpyAsync(s->tabs[d], tab.data(), bytes, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
      }
      s->ws_bytes += bytes;
    }
    if (prec == FLUPS_F64E) {
      // the double-float path reads a stored spectrum: evaluate the closed form in FP64 once
      int gext[3];
      long long n = 1;
      for (int d = 0; d < 3; ++d) {
        gext[d] = s->dir[d].gext;
        n *= gext[d];
      }
      double* g64 = nullptr;
      CK(cudaMallocAsync(&g64, n * sizeof(double), st));
      const double* tabs[3] = {(const double*)s->tabs[0], (const double*)s->tabs[1], (const double*)s->tabs[2]};
      cudaError_t e = launch_green_spectral(g64, gext, tabs, s->green, 0.5 * s->eps * s->eps, 1.0 / Pprod, st);
      s->green_pitch = (gext[0] + 1) & ~1;  // 16-byte rows (8-byte elements)
      const size_t padded = (size_t)s->green_pitch * gext[1] * gext[2] * 8;
      if (!e) e = cudaMallocAsync(&s->green_dev, padded, st);
      if (!e) e = launch_green_finalize(g64, s->green_dev, prec, n, gext[0], s->green_pitch, 1.0, st);
      cudaFreeAsync(g64, st);
      cudaError_t e2 = cudaStreamSynchronize(st);
      if (e || e2) return cuda_fail(e ? e : e2, "green spectral");
      s->green_bytes = (double)n * 8;
      s->ws_bytes += padded;
    }
    return FLUPS_OK;
  }
  // stored spectrum: sample G(k_s, r_u) in FP64, DCT-I along each unbounded-like direction
  GreenSampleParams q = green_params(s);
  long long n = 1;
  for (int d = 0; d < 3; ++d) n *= q.gext[d];
  double* g64 = nullptr;
  CK(cudaMallocAsync(&g64, n * sizeof(double), st));
  cudaError_t e = sample_green(s, q, g64, st);
  if (e) { cudaFreeAsync(g64, st); return cuda_fail(e, "green sample"); }
  double vol = 1.0;
  for (int d = 0; d < 3; ++d) {
    const DirPlan& dp = s->dir[d];
    if (!dp.unb) continue;
    vol *= dp.h;
    // node-centred even-even forward pass on M+1 samples: the DCT-I of the symmetrised kernel
    DirPlan gp{};
    gp.type = T_EE;
    gp.n_data = dp.gext;
    gp.N = dp.gext - 1;
    gp.P = 2 * gp.N;
    gp.nm = dp.gext;
    gp.rp = radix_plan(gp.P);
    // in double-float arithmetic on the FP32 units (FP64 samples in and out, ~1e-14 relative):
    // GB300's FP64 units would make these passes the bulk of a plan's setup time
    int rc = make_twiddles(gp.P, FLUPS_F64E, &gp.tw);
    if (rc) { cudaFreeAsync(g64, st); return rc; }
    Launch L{};
    L.kind = K_FWD_REAL;
    fill_geom(L, gp, d, q.gext, q.gext, FLUPS_F64E, true, FLUPS_NODE, 1);
    L.p.in = g64;
    L.p.out = g64;
    L.p.in_f64 = 1;
    L.p.out_f64 = 1;
    e = launch_pass(L.kind, FLUPS_F64E, L.p, L.grid, L.nthr, L.smem, st);
    if (e) { cudaFreeAsync(g64, st); return cuda_fail(e, "green DCT-I"); }
  }
  const double scale = vol / Pprod;
  const size_t bytes = n * esize(prec);
  // x rows padded to 16 bytes (TMA tensor maps need 16-byte strides)
  const int per16 = (int)(16 / esize(prec));
  s->green_pitch = (q.gext[0] + per16 - 1) / per16 * per16;
  const size_t padded = (size_t)s->green_pitch * q.gext[1] * q.gext[2] * esize(prec);
  e = cudaMallocAsync(&s->green_dev, padded, st);
  if (e) { cudaFreeAsync(g64, st); return cuda_fail(e, "green alloc"); }
  e = launch_green_finalize(g64, s->green_dev, prec, n, q.gext[0], s->green_pitch, scale, st);
  cudaFreeAsync(g64, st);
  cudaError_t e2 = cudaStreamSynchronize(st);
  if (e || e2) return cuda_fail(e ? e : e2, "green finalize");
  s->green_bytes = (double)bytes;
  s->ws_bytes += padded;
  return FLUPS_OK;
}

// Stored spectra shared between solvers (the serving runtime): solvers whose spectra are the same
// data -- same device, precision, kernel, eps and, per direction, the same sampling (unbounded-
// like: gext, P, h) or wavenumbers (spectral: gext, P, wscale, wshift) -- hold one device copy.
// Solvers opt in (flups_solver_share_green); the last one released frees it, stream-ordered on its
// release stream, which is safe when no solve of any sharing solver is still in flight (the
// serving runtime releases idle plans only).
struct GreenEntry {
  void* dev;
  int pitch;
  double bytes;
  size_t padded;
  int refs;
};
std::mutex g_green_mu;
std::map<std::string, GreenEntry> g_green_cache;

std::string green_cache_key(const flups_solver_s* s) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::string k;
  auto put = [&](const void* p, size_t n) { k.append((const char*)p, n); };
  put(&dev, sizeof dev);
  put(&s->topo.prec, sizeof s->topo.prec);
  put(&s->green, sizeof s->green);
  put(&s->eps, sizeof s->eps);
  for (int d = 0; d < 3; ++d) {
    const DirPlan& dp = s->dir[d];
    put(&dp.unb, sizeof dp.unb);
    put(&dp.gext, sizeof dp.gext);
    put(&dp.P, sizeof dp.P);
    put(&dp.h, sizeof dp.h);
    if (!dp.unb) {
      put(&dp.wscale, sizeof dp.wscale);
      put(&dp.wshift, sizeof dp.wshift);
    }
  }
  return k;
}

int setup_green(flups_solver_s* s, cudaStream_t st) {
  int du = 0;
  for (int d = 0; d < 3; ++d) du += s->dir[d].unb;
  const bool stored = du > 0 || s->topo.prec == FLUPS_F64E;
  if (!s->share_green || !stored) return setup_green_compute(s, st);
  const std::string key = green_cache_key(s);
  {
    std::lock_guard<std::mutex> lk(g_green_mu);
    auto it = g_green_cache.find(key);
    if (it != g_green_cache.end()) {
      it->second.refs++;
      s->green_dev = it->second.dev;
      s->green_pitch = it->second.pitch;
      s->green_bytes = it->second.bytes;
      s->green_key = key;
      return FLUPS_OK;
    }
  }
  const int rc = setup_green_compute(s, st);
  if (rc || !s->green_dev) return rc;
  std::lock_guard<std::mutex> lk(g_green_mu);
  auto it = g_green_cache.find(key);
  if (it != g_green_cache.end()) {
    // another solver stored the same spectrum meanwhile: use that copy
    cudaFreeAsync(s->green_dev, st);
    it->second.refs++;
    s->green_dev = it->second.dev;
    s->green_pitch = it->second.pitch;
  } else {
    const size_t padded = (size_t)s->green_pitch * s->dir[1].gext * s->dir[2].gext * esize(s->topo.prec);
    g_green_cache[key] = GreenEntry{s->green_dev, s->green_pitch, s->green_bytes, padded, 1};
  }
  s->green_key = key;
  return FLUPS_OK;
}

int build_plan(flups_solver_s* s) {
  const int center = s->topo.center;
  // per-direction geometry
  for (int d = 0; d < 3; ++d) {
    DirPlan& dp = s->dir[d];
    dp.type = s->types[d];
    dp.n_data = s->topo.n[d];
    // N = L / h; the stored count must be N (cell), N + 1 (node), or N for a
    // node-centred periodic direction given without its duplicate node
    const double ratio = s->L[d] / s->h[d];
    const long Nh = std::lround(ratio);
    if (std::fabs(ratio - (double)Nh) > 1e-6 * ratio) return FLUPS_ESIZE;
    if (center == FLUPS_CELL) {
      if (dp.n_data != Nh) return FLUPS_ESIZE;
    } else if (!(dp.n_data == Nh + 1 || (dp.type == T_PER && dp.n_data == Nh))) {
      return FLUPS_ESIZE;
    }
    dp.N = (int)Nh;
    if (!is_2a3b(dp.N) || dp.N < 4) return FLUPS_ESIZE;
    const int t = dp.type;
    dp.P = t == T_PER ? dp.N : ((t == T_UNB || t == T_EE || t == T_OO) ? 2 * dp.N : 4 * dp.N);
    if (dp.P > 4096) return FLUPS_ESIZE;
    dp.h = s->h[d];
    dp.L = s->L[d];
    dp.unb = is_unb_like(t);
    if (t == T_PER) { dp.gext = dp.N / 2 + 1; dp.wscale = 2.0 * M_PI / dp.L; dp.wshift = 0.0; }
    else if (t == T_UNB) { dp.gext = dp.N + 1; }
    else if (is_semi_t(t)) { dp.gext = 2 * dp.N + 1; }
    else if (is_quarter_t(t)) { dp.gext = dp.N; dp.wscale = M_PI / dp.L; dp.wshift = 0.5; }
    else { dp.gext = dp.N + 1; dp.wscale = M_PI / dp.L; dp.wshift = 0.0; }
    dp.rp = radix_plan(dp.P);
  }
  // order by cost, ties in x, y, z order
  int ord[3] = {0, 1, 2};
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (cost_class(s->dir[ord[j]].type) < cost_class(s->dir[ord[i]].type) ||
          (cost_class(s->dir[ord[j]].type) == cost_class(s->dir[ord[i]].type) && ord[j] < ord[i])) {
        int tmp = ord[i]; ord[i] = ord[j]; ord[j] = tmp;
      }
  for (int i = 0; i < 3; ++i) s->order[i] = ord[i];
  // roles and mode counts
  bool real = true;
  for (int i = 0; i < 3; ++i) {
    DirPlan& dp = s->dir[ord[i]];
    const int t = dp.type;
    if (t == T_PER || t == T_UNB) {
      if (real) { dp.role = R_R2C; dp.nm = dp.P / 2 + 1; real = false; }
      else { dp.role = R_C2C; dp.nm = dp.P; }
    } else {
      dp.role = R_R2R;
      dp.nm = is_semi_t(t) ? 2 * dp.N + 1 : (is_quarter_t(t) ? dp.N : dp.N + 1);
    }
  }
  // array dims after each forward pass (the fused direction keeps its data size)
  for (int d = 0; d < 3; ++d) s->dims[0][d] = s->topo.n[d];
  s->cplx[0] = 0;
  for (int i = 0; i < 2; ++i) {
    const DirPlan& dp = s->dir[ord[i]];
    for (int d = 0; d < 3; ++d) s->dims[i + 1][d] = s->dims[i][d];
    s->dims[i + 1][ord[i]] = dp.nm;
    s->cplx[i + 1] = s->cplx[i] || dp.role != R_R2R;
  }
  // x pitch of each array: the caller's arrays are dense; the workspaces' rows are padded to
  // 16 bytes so that TMA tensor maps can describe them
  s->pitch[0] = s->dims[0][0];
  for (int i = 1; i <= 2; ++i) {
    const int elem = (s->cplx[i] ? 2 : 1) * (s->topo.prec == FLUPS_F32 ? 4 : 8);
    const int per16 = elem >= 16 ? 1 : 16 / elem;
    s->pitch[i] = (s->dims[i][0] + per16 - 1) / per16 * per16;
  }
  return FLUPS_OK;
}

// A caller-provided workspace ends with a 256-byte block whose first int is the device status
// word of the solve that uses it (zeroed at the start of the solve, set by a bounded wait that
// gives up), so that concurrent solves of one plan report their device status separately.
constexpr size_t kStatusBlock = 256;

// Bytes of workspace array i (1: after d1, 2: after d2), padded rows, rounded to 256.
size_t ws_array_bytes(const flups_solver_s* s, int i) {
  return (((size_t)s->pitch[i] * s->dims[i][1] * s->dims[i][2] * s->topo.ncomp * (s->cplx[i] ? 2 : 1) *
           (s->topo.prec == FLUPS_F32 ? 4 : 8)) + 255) & ~(size_t)255;
}

// TMA tensor maps of the stored Green spectrum for the fused column pass: a 3D map (x, y, z) with
// the x rows at the spectrum's 16-byte pitch; map 0 has boxes of W lanes x gbox rows along the
// fused axis, map 1 boxes of W lanes x 1 row (the last folded mode P/2).  The encoder comes from
// the driver through the runtime's entry-point query, so the library links no driver library.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    cudaGetLastError();
  });
  return fn;
}

// Encodes both maps into the solver's device buffer; false (and no maps) when TMA does not apply.
bool green_tensor_maps(flups_solver_s* s, int axis, int W, int P, int prec, int* gbox, cudaStream_t st) {
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc || !s->green_dev || axis == 0) return false;
  const size_t es = esize(prec);
  if ((W * es) % 16 != 0 || (s->green_pitch * es) % 16 != 0) return false;
  const int rb = std::min(256, P / 2);
  if ((P / 2) % rb != 0) return false;
  cuuint64_t dims[3], strides[2];
  for (int d = 0; d < 3; ++d) dims[d] = (cuuint64_t)s->dir[d].gext;
  strides[0] = (cuuint64_t)s->green_pitch * es;
  strides[1] = strides[0] * (cuuint64_t)s->dir[1].gext;
  const CUtensorMapDataType dt = prec == FLUPS_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  const cuuint32_t estr[3] = {1, 1, 1};
  CUtensorMap maps[2];
  for (int m = 0; m < 2; ++m) {
    const cuuint32_t rows = m == 0 ? (cuuint32_t)rb : 1u;
    const cuuint32_t box[3] = {(cuuint32_t)W, axis == 1 ? rows : 1u, axis == 2 ? rows : 1u};
    if (enc(&maps[m], dt, 3, s->green_dev, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  if (!s->gmaps_dev && cudaMallocAsync(&s->gmaps_dev, sizeof(maps), st) != cudaSuccess) {
    cudaGetLastError();
    s->gmaps_dev = nullptr;
    return false;
  }
  if (cudaMemcpyAsync(s->gmaps_dev, maps, sizeof(maps), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  *gbox = rb;
  return true;
}

// TMA map of a column pass's input array (the T2 variant of a direction change: the tile arrives
// by bulk tensor copies instead of per-thread loads).  4D: x in 8-byte units (one FP32 complex,
// half an FP64 or double-float complex), y, z, component; the axis exposes the rows the pass reads
// (n_use forward, P inverse; rows beyond arrive as zeros); boxes of W lanes x up to 256 rows.
// Leaves p.tin_rows = 0 (per-thread loads) when the pass or the array does not qualify.
void encode_input_map(Launch& L, int prec) {
  PassParams& p = L.p;
  p.tin_rows = 0;
  const bool col = p.ct && p.axis != 0 && (L.kind == K_FWD_C2C || L.kind == K_INV_C2C || L.kind == K_FUSED_C2C);
  EncodeTiledFn enc = tensor_map_encoder();
  if (!col || !enc || !p.in) return;
  const size_t cb = 2 * esize(prec);
  const cuuint64_t u = cb / 8;
  const bool inv = L.kind == K_INV_C2C;
  const int n_in = inv ? p.P : p.n_use;
  const int rows = (p.hz && !inv) ? p.P / 2 : p.P;
  const int box = std::min(256, rows);
  if (n_in > rows || rows % box != 0 || ((size_t)p.W * cb) % 16 != 0) return;
  // measured: FP32 tiles gain at every length (unbounded 512^3: y inverse -15%, fused -4%); FP64 and
  // double-float tiles gain with 128-byte rows (P <= 512) and lose with narrower ones (P = 1024:
  // column passes +6..17%), where the per-thread loads overlap the first stage better
  if (prec != FLUPS_F32 && (size_t)p.W * cb < 128) return;
  const bool ax1 = p.axis == 1;
  const cuuint64_t dims[4] = {(cuuint64_t)p.npen * u, (cuuint64_t)(ax1 ? n_in : (int)L.grid.y),
                              (cuuint64_t)(ax1 ? (int)L.grid.y : n_in), (cuuint64_t)L.grid.z};
  const cuuint64_t strides[3] = {(cuuint64_t)((ax1 ? p.ai.js : p.ai.os) * cb),
                                 (cuuint64_t)((ax1 ? p.ai.os : p.ai.js) * cb), (cuuint64_t)(p.ai.cs * cb)};
  for (int d = 0; d < 3; ++d)
    if (strides[d] % 16 != 0) return;
  const cuuint32_t boxd[4] = {(cuuint32_t)(p.W * u), ax1 ? (cuuint32_t)box : 1u, ax1 ? 1u : (cuuint32_t)box, 1u};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  if (enc(&p.tin, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, const_cast<void*>(p.in), dims, strides, boxd, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return;
  p.tin_rows = rows;
  p.tin_box = box;
}

// x passes of periodic or doubled unbounded cell-centred real data in 4-lane FP32 tiles run on the
// column kernels' register-chained stages (k_fwd_rowx, k_inv_rowx): the generic row kernels spent
// about 100-120 instructions per element on one transform and half their shared-memory
// wavefronts on bank conflicts (unbounded 512x256x256 FP32 under ncu).
void set_rowx(Launch& L, int prec) {
  PassParams& p = L.p;
  p.rowx = 0;
  if (!p.ct || p.axis != 0 || (prec != FLUPS_F32 && prec != FLUPS_F64E) || p.W != 4 || p.center != C_CELL) return;
  if (L.kind != K_FWD_REAL && L.kind != K_INV_REAL) return;
  for (int c = 0; c < (int)L.grid.z; ++c) {
    const int t = (p.ctypes >> (4 * c)) & 15;
    if (!((t == T_UNB && 2 * p.n_data == p.P) || (t == T_PER && p.n_data == p.P))) return;
  }
  L.gnthr = L.nthr;
  L.gsmem = L.smem;
  p.rowx = 1;
  // measured at 512^3 (P = 1024): the forward pass runs best with 16 elements per thread (256
  // threads; 0.488 vs 0.516 ms with radix-32 stages), the inverse with radix-32 stages and its
  // rows staged by a bulk copy (0.453 ms; 0.492 with 16 elements per thread)
  p.ept = (L.kind == K_FWD_REAL || prec != FLUPS_F32) ? 16 : ct_col_ept(p.P, prec, K_FWD_C2C);
  L.nthr = p.P * p.W / p.ept;
  L.smem = (size_t)p.P * (p.W + 1) * 2 * esize(prec) + 256;
}

// Inverse row pass (x) of complex modes: its CTA's 2W input rows, contiguous in memory, arrive in
// shared memory by one bulk copy instead of per-thread loads whose latency the pass could not hide
// (unbounded 512^3 FP32: long-scoreboard stalls were its largest).  Used where the rows are 16-byte
// aligned and the extra shared memory still leaves two CTAs per SM.
void set_rows_bulk(Launch& L, int prec) {
  PassParams& p = L.p;
  if (p.rows_bulk) {
    L.smem = p.rows_off - 128;  // back to the size without the staged rows
    p.rows_bulk = 0;
  }
  if (L.kind != K_INV_REAL || !p.ct || p.axis != 0 || prec != FLUPS_F32 || !p.in) return;
  for (int c = 0; c < 3; ++c) {
    const int t = (p.ctypes >> (4 * c)) & 15;
    if (t != T_PER && t != T_UNB) return;
  }
  const size_t cb = 2 * esize(prec);
  if (((uintptr_t)p.in % 16) != 0 || (p.ai.ls * cb) % 16 != 0 || (p.ai.cs * cb) % 16 != 0) return;
  const size_t off = ((L.smem + 15) & ~(size_t)15) + 128;  // 128 bytes for the mbarrier
  const size_t total = off + (size_t)2 * p.W * p.ai.ls * cb;
  if (2 * total > 227 * 1024) return;
  p.rows_off = (int)off;
  p.rows_bulk = 1;
  L.smem = total;
}

int build_passes(flups_solver_s* s, cudaStream_t st) {
  const int prec = s->topo.prec, center = s->topo.center, nc = s->topo.ncomp;
  const int* o = s->order;
  const size_t es = esize(prec);
  s->passes.clear();
  double bytes = 0.0;
  auto arr_bytes = [&](int i) {
    const double n = (double)s->dims[i][0] * s->dims[i][1] * s->dims[i][2];
    return n * es * (s->cplx[i] ? 2 : 1) * nc;
  };
  auto ffts = [&](const Launch& L, bool packed, int mult) {
    const double P = L.p.P;
    const double pencils = (double)L.p.npen * L.grid.y * nc;
    const double n = packed ? std::ceil(pencils / 2.0) : pencils;
    return mult * n * 5.0 * P * std::log2(P);
  };
  // 1: forward d1, user rhs -> W1
  {
    Launch L{};
    L.kind = K_FWD_REAL;
    fill_geom(L, s->dir[o[0]], o[0], s->dims[0], s->dims[1], prec, true, center, nc, 1, s->pitch[0], s->pitch[1]);
    L.p.ctypes = pack3(s->tf[0][o[0]], s->tf[1][o[0]], s->tf[2][o[0]]);
    L.p.out = s->W1;
    L.out_buf = 1;
    L.user_in = 1;
    L.p.in_f64 = prec == FLUPS_F64E;
    L.bytes = arr_bytes(0) + arr_bytes(1);
    L.flops = ffts(L, true, 1);
    s->passes.push_back(L);
    bytes += L.bytes;
  }
  // 2: forward d2, W1 -> W2
  {
    Launch L{};
    const bool real = !s->cplx[1];
    L.kind = real ? K_FWD_REAL : K_FWD_C2C;
    fill_geom(L, s->dir[o[1]], o[1], s->dims[1], s->dims[2], prec, real, center, nc, 1, s->pitch[1], s->pitch[2]);
    L.p.ctypes = pack3(s->tf[0][o[1]], s->tf[1][o[1]], s->tf[2][o[1]]);
    L.p.in = s->W1;
    L.p.out = s->W2;
    L.in_buf = 1;
    L.out_buf = 2;
    L.bytes = arr_bytes(1) + arr_bytes(2);
    L.flops = ffts(L, real, 1);
    s->passes.push_back(L);
    bytes += L.bytes;
  }
  // 3: fused d3 on W2, in place
  {
    Launch L{};
    const bool real = !s->cplx[2];
    const bool curl = s->op == FLUPS_BIOT_SAVART;
    L.kind = curl ? (real ? K_CURL_REAL : K_CURL_C2C) : (real ? K_FUSED_REAL : K_FUSED_C2C);
    const DirPlan& dp = s->dir[o[2]];
    fill_geom(L, dp, o[2], s->dims[2], s->dims[2], prec, real, center, curl ? 1 : nc, curl ? 3 : 1, s->pitch[2],
              s->pitch[2]);
    L.p.ctypes = pack3(s->tf[0][o[2]], s->tf[1][o[2]], s->tf[2][o[2]]);
    L.p.in = s->W2;
    L.p.out = s->W2;
    L.in_buf = 2;
    L.out_buf = 2;
    FusedGreen& g = L.p.g;
    if (curl) {
      L.smem = 6 * (size_t)dp.P * L.p.LS * 2 * esize(prec) + (size_t)(real ? 2 : 1) * L.p.W * (prec == FLUPS_F32 ? 96 : 176) + 16;
      g.utypes = pack3(s->tu[0][o[2]], s->tu[1][o[2]], s->tu[2][o[2]]);
      for (int d = 0; d < 3; ++d) {
        g.dsym[d] = s->dsym[d];
        g.role[d] = s->dir[d].role;
        g.quarter[d] = is_quarter_t(s->dir[d].type);
        g.srcodd[d] = 0;
        for (int c = 0; c < 3; ++c) {
          const int t = s->tf[c][d];
          if (t == T_OO || t == T_OE || t == T_OU || t == T_UO) g.srcodd[d] |= 1 << c;
        }
      }
    }
    g.stored = s->green_dev;
    for (int d = 0; d < 3; ++d) {
      g.tab[d] = s->tabs[d];
      g.gext[d] = s->dir[d].gext;
      g.fold[d] = (s->dir[d].role == R_C2C) ? s->dir[d].P : 0;
    }
    g.gpitch = s->green_dev ? s->green_pitch : s->dir[0].gext;
    if (!curl && !real && L.p.ct && o[2] != 0 && g.stored && dp.gext == dp.P / 2 + 1) {
      // register-chained fused column kernel: stage the tile's Green slice in shared memory
      // (cp.async at kernel start) when that keeps the kernel's CTAs per SM
      const size_t gbytes = (size_t)L.p.W * (dp.P / 2 + 1) * esize(prec);
      const int minb = ct_min_blocks(L.p, L.nthr, prec);
      if ((L.smem + gbytes + 128 + 1024) * minb <= 228 * 1024) {
        L.smem += gbytes + 128;  // + alignment of the slice to 128 bytes
        L.p.gpre = 1;
        // the slice by TMA when the lanes' x indices are contiguous in the spectrum (x not folded)
        if (g.fold[0] == 0 && green_tensor_maps(s, o[2], L.p.W, dp.P, prec, &L.p.gbox, st))
          L.p.gmap = s->gmaps_dev;
      }
    }
    g.kernel = s->green;
    g.eps2_half = 0.5 * s->eps * s->eps;
    g.scale = 1.0 / ((double)s->dir[0].P * s->dir[1].P * s->dir[2].P);
    g.quarter3 = is_quarter_t(dp.type);
    g.dims1 = s->dims[2][1];
    g.dims2 = s->dims[2][2];
    L.bytes = 2 * arr_bytes(2) + s->green_bytes;
    L.flops = ffts(L, real, 2);
    s->passes.push_back(L);
    bytes += L.bytes;
  }
  // 4: inverse d2, W2 -> W1
  {
    Launch L{};
    const bool real = !s->cplx[1];
    L.kind = real ? K_INV_REAL : K_INV_C2C;
    fill_geom(L, s->dir[o[1]], o[1], s->dims[2], s->dims[1], prec, real, center, nc, 1, s->pitch[2], s->pitch[1]);
    L.p.ctypes = pack3(s->tu[0][o[1]], s->tu[1][o[1]], s->tu[2][o[1]]);
    L.p.in = s->W2;
    L.p.out = s->W1;
    L.in_buf = 2;
    L.out_buf = 1;
    L.bytes = arr_bytes(1) + arr_bytes(2);
    L.flops = ffts(L, real, 1);
    s->passes.push_back(L);
    bytes += L.bytes;
  }
  // 5: inverse d1, W1 -> user phi
  {
    Launch L{};
    L.kind = K_INV_REAL;
    fill_geom(L, s->dir[o[0]], o[0], s->dims[1], s->dims[0], prec, true, center, nc, 1, s->pitch[1], s->pitch[0]);
    L.p.ctypes = pack3(s->tu[0][o[0]], s->tu[1][o[0]], s->tu[2][o[0]]);
    L.p.in = s->W1;
    L.in_buf = 1;
    L.user_out = 1;
    L.p.out_f64 = prec == FLUPS_F64E;
    L.bytes = arr_bytes(0) + arr_bytes(1);
    L.flops = ffts(L, true, 1);
    s->passes.push_back(L);
    bytes += L.bytes;
  }
  s->model_bytes = bytes;
  for (Launch& L : s->passes) set_rowx(L, prec);  // before set_rows_bulk (flups_setup): the staged rows follow the tile
  for (const Launch& L : s->passes)
    if (L.smem > 227 * 1024 || L.nthr > 1024) return FLUPS_ESIZE;
  return FLUPS_OK;
}

// Dynamic shared-memory limits of the pass and curl kernels: a per-device attribute, so it is set
// once for every device the library is used on, with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_limits_mu;
bool g_limits_done[kMaxDevices] = {};
cudaError_t g_limits_err[kMaxDevices] = {};

int ensure_smem_limits() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return FLUPS_EINVAL;
  std::lock_guard<std::mutex> lk(g_limits_mu);
  if (!g_limits_done[dev]) {
    cudaError_t e = set_pass_smem_limits();
    if (e == cudaSuccess) e = set_curl_smem_limits();
    g_limits_err[dev] = e;
    g_limits_done[dev] = true;
  }
  if (g_limits_err[dev] != cudaSuccess) return cuda_fail(g_limits_err[dev], "smem limits");
  return FLUPS_OK;
}

}  // namespace

namespace flups {
void host_gauss_legendre(int n, double* x, double* w) { gauss_legendre(n, x, w); }
}  // namespace flups

extern "C" {

const char* flups_strerror(int status) {
  switch (status) {
    case FLUPS_OK: return "ok";
    case FLUPS_EINVAL: return "invalid argument";
    case FLUPS_EBC: return "inadmissible boundary conditions";
    case FLUPS_ESIZE: return "unsupported grid size";
    case FLUPS_ENOMEM: return "out of memory";
    case FLUPS_ECUDA: return "CUDA error";
    case FLUPS_EGREEN: return "Green kernel not available for these boundary conditions";
    case FLUPS_ESTATE: return "call out of order";
    case FLUPS_EDEVICE: return "a kernel's bounded wait gave up: the result is not valid";
  }
  return "unknown status";
}

const char* flups_last_cuda_error(void) { return g_last_cuda.c_str(); }

int flups_init_topo(const int n[3], int center, int ncomp, int prec, flups_topo* out) {
  if (!n || !out) return FLUPS_EINVAL;
  if (center != FLUPS_CELL && center != FLUPS_NODE) return FLUPS_EINVAL;
  if (ncomp != 1 && ncomp != 3) return FLUPS_EINVAL;
  if (prec != FLUPS_F32 && prec != FLUPS_F64 && prec != FLUPS_F64E) return FLUPS_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (n[d] < 2 || n[d] > 8193) return FLUPS_ESIZE;
  flups_topo_s* t = new (std::nothrow) flups_topo_s;
  if (!t) return FLUPS_ENOMEM;
  for (int d = 0; d < 3; ++d) t->n[d] = n[d];
  t->center = center;
  t->ncomp = ncomp;
  t->prec = prec;
  *out = t;
  return FLUPS_OK;
}

int flups_topo_free(flups_topo t) {
  delete t;
  return FLUPS_OK;
}

int flups_init_solver(flups_topo t, const int* bc, const double h[3], const double L[3], int green,
                      double eps_over_h, int op, int diff, flups_solver* out) {
  if (!t || !bc || !h || !L || !out) return FLUPS_EINVAL;
  if (op != FLUPS_POISSON && op != FLUPS_BIOT_SAVART) return FLUPS_EINVAL;
  if (op == FLUPS_BIOT_SAVART && t->ncomp != 3) return FLUPS_EINVAL;
  if (op == FLUPS_BIOT_SAVART && !(diff == FLUPS_DIFF_SPECTRAL || diff == FLUPS_DIFF_FD2 || diff == FLUPS_DIFF_FD4 ||
                                   diff == FLUPS_DIFF_FD6))
    return FLUPS_EINVAL;
  const int gk[] = {FLUPS_SPECTRAL, FLUPS_HEJ0, FLUPS_HEJ2, FLUPS_HEJ4, FLUPS_HEJ6, FLUPS_HEJ8, FLUPS_HEJ10, FLUPS_LGF2};
  bool gok = false;
  for (int g : gk) gok |= (g == green);
  if (!gok) return FLUPS_EINVAL;
  if (!(eps_over_h > 0.0)) return FLUPS_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (!(h[d] > 0.0) || !(L[d] > 0.0)) return FLUPS_EINVAL;
  flups_solver_s* s = new (std::nothrow) flups_solver_s;
  if (!s) return FLUPS_ENOMEM;
  s->topo = *t;
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d)
      for (int f = 0; f < 2; ++f) s->bc[c][d][f] = c < t->ncomp ? bc[(c * 3 + d) * 2 + f] : bc[(d * 2) + f];
  for (int d = 0; d < 3; ++d) {
    s->h[d] = h[d];
    s->L[d] = L[d];
  }
  s->green = green;
  s->op = op;
  s->diff = diff;
  s->eps_over_h = eps_over_h;
  s->eps = eps_over_h * std::fmax(h[0], std::fmax(h[1], h[2]));
  int rc = FLUPS_OK;
  for (int c = 0; c < t->ncomp && rc == FLUPS_OK; ++c)
    for (int d = 0; d < 3 && rc == FLUPS_OK; ++d) rc = classify(s->bc[c][d][0], s->bc[c][d][1], &s->tf[c][d]);
  for (int c = t->ncomp; c < 3; ++c)
    for (int d = 0; d < 3; ++d) s->tf[c][d] = s->tf[0][d];
  for (int d = 0; d < 3; ++d) s->types[d] = s->tf[0][d];
  if (rc == FLUPS_OK && op == FLUPS_POISSON) {
    // a vector Poisson solve shares one plan: every component needs the same conditions
    for (int c = 1; c < t->ncomp && rc == FLUPS_OK; ++c)
      for (int d = 0; d < 3; ++d)
        if (s->bc[c][d][0] != s->bc[0][d][0] || s->bc[c][d][1] != s->bc[0][d][1]) rc = FLUPS_EBC;
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) s->tu[c][d] = s->tf[c][d];
  }
  if (rc == FLUPS_OK && op == FLUPS_BIOT_SAVART) {
    // one geometry per direction for the three components
    for (int d = 0; d < 3 && rc == FLUPS_OK; ++d)
      for (int c = 1; c < 3; ++c)
        if (family(s->tf[c][d]) != family(s->tf[0][d])) rc = FLUPS_EBC;
    // u_c = d_a f_b - d_b f_a: along d each term keeps its source's faces, with
    // even/odd swapped along the differentiated direction; both terms must agree
    for (int c = 0; c < 3 && rc == FLUPS_OK; ++c) {
      const int a = (c + 1) % 3, b = (c + 2) % 3;
      for (int d = 0; d < 3 && rc == FLUPS_OK; ++d) {
        int f1[2], f2[2];
        for (int f = 0; f < 2; ++f) {
          f1[f] = d == a ? swap_parity(s->bc[b][d][f]) : s->bc[b][d][f];
          f2[f] = d == b ? swap_parity(s->bc[a][d][f]) : s->bc[a][d][f];
        }
        if (f1[0] != f2[0] || f1[1] != f2[1]) rc = FLUPS_EBC;
        else rc = classify(f1[0], f1[1], &s->tu[c][d]);
      }
    }
  }
  if (rc == FLUPS_OK) rc = build_plan(s);
  if (rc == FLUPS_OK) {
    int du = 0;
    for (int d = 0; d < 3; ++d) du += s->dir[d].unb;
    if (du == 0 && green == FLUPS_HEJ0) rc = FLUPS_EGREEN;
    const bool hej2m = green >= FLUPS_HEJ2 && green <= FLUPS_HEJ10;
    if (du > 0 && !(hej2m || ((green == FLUPS_HEJ0 || green == FLUPS_LGF2) && du == 3))) rc = FLUPS_EGREEN;
  }
  if (rc != FLUPS_OK) {
    delete s;
    return rc;
  }
  *out = s;
  return FLUPS_OK;
}

int flups_setup(flups_solver s, void* stream, size_t* workspace_bytes) {
  if (!s) return FLUPS_EINVAL;
  if (s->ready) {
    if (workspace_bytes) *workspace_bytes = s->ws_bytes;
    return FLUPS_OK;
  }
  {
    const int rc = ensure_smem_limits();
    if (rc) return rc;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int prec = s->topo.prec, nc = s->topo.ncomp;
  const size_t es = esize(prec);
  if (s->op == FLUPS_BIOT_SAVART) {
    for (int d = 0; d < 3; ++d) {
      int rc = make_dsym(s->dir[d].P, s->dir[d].h, s->diff, prec, &s->dsym[d], st);
      if (rc) return rc;
      s->ws_bytes += (size_t)s->dir[d].P * es;
    }
  }
  for (int d = 0; d < 3; ++d) {
    int rc = make_twiddles(s->dir[d].P, prec, &s->dir[d].tw);
    if (rc) return rc;
    s->ws_bytes += (size_t)4 * s->dir[d].P * es;
  }
  size_t wbytes[3] = {0, 0, 0};
  for (int i = 1; i <= 2; ++i) wbytes[i] = ws_array_bytes(s, i);
  s->ws_need = wbytes[1] + wbytes[2] + kStatusBlock;
  if (!s->shared) {
    for (int i = 1; i <= 2; ++i) {
      void** buf = i == 1 ? &s->W1 : &s->W2;
      cudaError_t e = cudaMallocAsync(buf, wbytes[i], st);
      if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return FLUPS_ENOMEM;
      }
      if (e) return cuda_fail(e, "workspace alloc");
      s->ws_bytes += wbytes[i];
    }
  }
  if (!s->errflag) {
    CK(cudaMallocAsync((void**)&s->errflag, sizeof(int), st));
    CK(cudaMemsetAsync(s->errflag, 0, sizeof(int), st));
  }
  int rc = setup_green(s, st);
  if (rc) return rc;
  rc = build_passes(s, st);
  if (rc) return rc;
  for (Launch& L : s->passes) {
    L.p.errflag = s->errflag;
    encode_input_map(L, prec);
    set_rows_bulk(L, prec);
  }
  CK(cudaStreamSynchronize(st));
  s->user_bytes = (size_t)s->topo.n[0] * s->topo.n[1] * s->topo.n[2] * nc * es;
  s->ready = true;
  if (workspace_bytes) *workspace_bytes = s->ws_bytes;
  return FLUPS_OK;
}

// Launch the whole pass list with the given workspace (W1 at ws, W2 after it).  host_in / host_out:
// rhs / phi are pinned host memory read or written by the kernels across the host link; the x
// passes then run the generic row kernels, whose warps touch 128 contiguous bytes of one row (the
// register-chained ones touch 32-byte pieces of 8 rows, which the link serves less well).
static int solve_impl(flups_solver s, void* phi, const void* rhs, void* ws, void* stream, bool host_in = false,
                      bool host_out = false) {
  cudaStream_t st = (cudaStream_t)stream;
  const int prec = s->topo.prec;
  void* W[3] = {nullptr, s->W1, s->W2};
  int* status = s->errflag;
  if (ws) {
    const size_t w1 = ws_array_bytes(s, 1);
    W[1] = ws;
    W[2] = (char*)ws + w1;
    status = (int*)((char*)ws + s->ws_need - kStatusBlock);
    CK(cudaMemsetAsync(status, 0, sizeof(int), st));
  }
  auto launch_one = [&](const Launch& L) -> int {
    Launch Lw = L;
    PassParams& p = Lw.p;
    p.errflag = status;
    p.dbg_wait = s->dbg_wait;
    p.pdl = 1;  // each pass a programmatic dependent of the stream's previous kernel
    if (L.in_buf) p.in = W[L.in_buf];
    if (L.out_buf) p.out = W[L.out_buf];
    if (L.user_in) p.in = rhs;
    if (L.user_out) p.out = phi;
    if (ws && L.in_buf) {  // the caller's workspace: maps and alignment of its addresses
      encode_input_map(Lw, prec);
      set_rows_bulk(Lw, prec);
    }
    if (p.rowx && ((L.user_in && host_in) || (L.user_out && host_out))) {
      p.rowx = 0;
      Lw.nthr = L.gnthr;
      if (!p.rows_bulk) Lw.smem = L.gsmem;
    }
    cudaError_t e = L.kind >= K_CURL_REAL ? launch_curl(L.kind, prec, p, Lw.grid, Lw.nthr, Lw.smem, st)
                                          : launch_pass(L.kind, prec, p, Lw.grid, Lw.nthr, Lw.smem, st);
    if (e) return cuda_fail(e, "pass launch");
    return FLUPS_OK;
  };
  for (const Launch& L : s->passes) {
    const int rc = launch_one(L);
    if (rc) return rc;
  }
  return FLUPS_OK;
}

int flups_solve(flups_solver s, void* phi, const void* rhs, void* stream) {
  if (!s || !phi || !rhs) return FLUPS_EINVAL;
  if (!s->ready) return FLUPS_ESTATE;
  if (s->shared) return FLUPS_ESTATE;  // no own workspace: use flups_solve_ws
  return solve_impl(s, phi, rhs, nullptr, stream);
}

int flups_solver_memory(flups_solver s, size_t* resident, size_t* transient, size_t* workspace) {
  if (!s) return FLUPS_EINVAL;
  const int prec = s->topo.prec, nc = s->topo.ncomp;
  const size_t es = esize(prec);
  size_t res = 0, tr = 0, ws = 0;
  int du = 0;
  size_t gn = 1, gmax = 0;
  for (int d = 0; d < 3; ++d) {
    res += (size_t)4 * s->dir[d].P * es;  // twiddles
    du += s->dir[d].unb;
    gn *= (size_t)s->dir[d].gext;
    if ((size_t)s->dir[d].gext > gmax) gmax = s->dir[d].gext;
    if (s->op == FLUPS_BIOT_SAVART) res += (size_t)s->dir[d].P * es;
  }
  if (du == 0) {
    for (int d = 0; d < 3; ++d) res += (size_t)s->dir[d].gext * es;
  } else {
    res += gn * es;
    tr += gn * sizeof(double) + (size_t)8 * 2 * gmax * sizeof(double);
  }
  for (int i = 1; i <= 2; ++i) ws += ws_array_bytes(s, i);
  ws += kStatusBlock;
  if (resident) *resident = res;
  if (transient) *transient = tr;
  if (workspace) *workspace = ws;
  return FLUPS_OK;
}

int flups_workspace_size(flups_solver s, size_t* bytes) {
  if (!s || !bytes) return FLUPS_EINVAL;
  if (!s->ready) return FLUPS_ESTATE;
  *bytes = s->ws_need;
  return FLUPS_OK;
}

int flups_workspace_status(flups_solver s, size_t* offset) {
  if (!s || !offset) return FLUPS_EINVAL;
  if (!s->ready) return FLUPS_ESTATE;
  *offset = s->ws_need - kStatusBlock;
  return FLUPS_OK;
}

int flups_debug_green(flups_solver s, double* samples, double* spectrum, long long n) {
  if (!s || !samples || !spectrum) return FLUPS_EINVAL;
  if (!s->ready) return FLUPS_ESTATE;
  int du = 0;
  for (int d = 0; d < 3; ++d) du += s->dir[d].unb;
  if (du == 0 || !s->green_dev) return FLUPS_ESTATE;  // closed form: no stored spectrum
  GreenSampleParams q = green_params(s);
  const long long cnt = (long long)q.gext[0] * q.gext[1] * q.gext[2];
  if (n != cnt) return FLUPS_EINVAL;
  double* g64 = nullptr;
  CK(cudaMalloc(&g64, cnt * sizeof(double)));
  cudaError_t e = sample_green(s, q, g64, nullptr);
  if (!e) e = cudaMemcpy(samples, g64, cnt * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(g64);
  if (e) return cuda_fail(e, "flups_debug_green samples");
  const size_t es = s->topo.prec == FLUPS_F32 ? 4 : 8;
  const size_t rows = (size_t)q.gext[1] * q.gext[2];
  std::vector<unsigned char> buf(rows * s->green_pitch * es);
  CK(cudaMemcpy(buf.data(), s->green_dev, buf.size(), cudaMemcpyDeviceToHost));
  // element formats: FP32, FP64, or on the double-float path a pair of floats (hi, lo)
  for (size_t r = 0; r < rows; ++r)
    for (int x = 0; x < q.gext[0]; ++x) {
      const size_t i = r * s->green_pitch + x;
      double v;
      if (es == 4) v = (double)((const float*)buf.data())[i];
      else if (s->topo.prec == FLUPS_F64E) v = (double)((const float*)buf.data())[2 * i] + (double)((const float*)buf.data())[2 * i + 1];
      else v = ((const double*)buf.data())[i];
      spectrum[r * q.gext[0] + x] = v;
    }
  return FLUPS_OK;
}

int flups_debug_wait_limit(flups_solver s, int mask) {
  if (!s || mask < 0 || mask > 3) return FLUPS_EINVAL;
  s->dbg_wait = mask;
  return FLUPS_OK;
}

int flups_setup_shared(flups_solver s, void* stream) {
  if (!s) return FLUPS_EINVAL;
  if (s->ready) return s->shared ? FLUPS_OK : FLUPS_ESTATE;
  s->shared = true;
  return flups_setup(s, stream, nullptr);
}

int flups_solve_ws(flups_solver s, void* phi, const void* rhs, void* workspace, void* stream) {
  if (!s || !phi || !rhs || !workspace) return FLUPS_EINVAL;
  if (!s->ready) return FLUPS_ESTATE;
  if (((uintptr_t)workspace & 255) != 0) return FLUPS_EINVAL;
  return solve_impl(s, phi, rhs, workspace, stream);
}

int flups_solve_pass(flups_solver s, int i, void* phi, const void* rhs, void* stream) {
  if (!s || !phi || !rhs) return FLUPS_EINVAL;
  if (!s->ready || s->shared) return FLUPS_ESTATE;
  if (i < 0 || i >= (int)s->passes.size()) return FLUPS_EINVAL;
  const Launch& L = s->passes[i];
  PassParams p = L.p;
  p.dbg_wait = s->dbg_wait;
  if (L.user_in) p.in = rhs;
  if (L.user_out) p.out = phi;
  cudaError_t e = L.kind >= K_CURL_REAL
                      ? launch_curl(L.kind, s->topo.prec, p, L.grid, L.nthr, L.smem, (cudaStream_t)stream)
                      : launch_pass(L.kind, s->topo.prec, p, L.grid, L.nthr, L.smem, (cudaStream_t)stream);
  if (e) return cuda_fail(e, "pass launch");
  return FLUPS_OK;
}

int flups_solve_events(flups_solver s, void* phi, const void* rhs, void* stream, void* const* events) {
  if (!s || !phi || !rhs || !events) return FLUPS_EINVAL;
  if (!s->ready || s->shared) return FLUPS_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  const int n = (int)s->passes.size();
  for (int i = 0; i < n; ++i) {
    CK(cudaEventRecord((cudaEvent_t)events[i], st));
    const int rc = flups_solve_pass(s, i, phi, rhs, stream);
    if (rc) return rc;
  }
  CK(cudaEventRecord((cudaEvent_t)events[n], st));
  return FLUPS_OK;
}

int flups_pass_info(flups_solver s, int i, int* kind, int* axis, int* fft_len, double* bytes, double* flops) {
  if (!s) return FLUPS_EINVAL;
  if (!s->ready) return FLUPS_ESTATE;
  if (i < 0 || i >= (int)s->passes.size()) return FLUPS_EINVAL;
  const Launch& L = s->passes[i];
  if (kind) *kind = L.kind;
  if (axis) *axis = L.p.axis;
  if (fft_len) *fft_len = L.p.P;
  if (bytes) *bytes = L.bytes;
  if (flops) *flops = L.flops;
  return FLUPS_OK;
}

int flups_pass_features(flups_solver s, int i, int* flags) {
  if (!s || !flags) return FLUPS_EINVAL;
  if (!s->ready) return FLUPS_ESTATE;
  if (i < 0 || i >= (int)s->passes.size()) return FLUPS_EINVAL;
  const PassParams& p = s->passes[i].p;
  *flags = (p.ct ? 1 : 0) | (p.gpre ? 2 : 0) | (p.gmap ? 4 : 0) | (p.hz ? 8 : 0) | (p.tin_rows ? 16 : 0) |
           (p.rowx ? 32 : 0) | (p.rows_bulk ? 64 : 0);
  return FLUPS_OK;
}

// Device address of a host range [p, p + bytes) that the device can load from and store to
// directly: pinned memory (cudaHostAlloc, cudaHostRegister), mapped into the unified address
// space, checked at both ends of the range.  nullptr for pageable memory or a range that leaves
// its pinned allocation.
static void* mapped_device_ptr(const void* p, size_t bytes) {
  if (!p || bytes == 0) return nullptr;
  cudaPointerAttributes a{}, b{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  const char* last = (const char*)p + (bytes - 1);
  if (cudaPointerGetAttributes(&b, last) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (b.type != cudaMemoryTypeHost || (const char*)b.devicePointer != (const char*)a.devicePointer + (bytes - 1))
    return nullptr;
  return a.devicePointer;
}

int flups_host_mapped(const void* host, size_t bytes) { return mapped_device_ptr(host, bytes) ? 1 : 0; }

int flups_solve_host(flups_solver s, void* phi_host, const void* rhs_host, void* stream) {
  if (!s || !phi_host || !rhs_host) return FLUPS_EINVAL;
  if (!s->ready || s->shared) return FLUPS_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  // Pinned arrays are used in place: the first pass loads rhs and the last pass stores phi across
  // the host link, so the transfers run inside the two x passes instead of before and after them.
  const void* rin = mapped_device_ptr(rhs_host, s->user_bytes);
  void* rout = mapped_device_ptr(phi_host, s->user_bytes);
  if ((!rin || !rout) && !s->stage) {
    cudaError_t e = cudaMalloc(&s->stage, s->user_bytes);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      return FLUPS_ENOMEM;
    }
    if (e) return cuda_fail(e, "stage alloc");
    s->ws_bytes += s->user_bytes;
  }
  if (!rin) {
    CK(cudaMemcpyAsync(s->stage, rhs_host, s->user_bytes, cudaMemcpyHostToDevice, st));
    rin = s->stage;
  }
  int rc = solve_impl(s, rout ? rout : s->stage, rin, nullptr, stream, rin != s->stage, rout != nullptr);
  if (rc) return rc;
  if (!rout) CK(cudaMemcpyAsync(phi_host, s->stage, s->user_bytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return FLUPS_OK;
}

// Frees the solver's own device buffers on `st` (stream-ordered) or, with
// st == nullptr, synchronously.  Twiddle tables are shared and stay.
static void release(flups_solver s, cudaStream_t st, bool async) {
  auto fr = [&](void* p) {
    if (!p) return;
    if (async) cudaFreeAsync(p, st);
    else cudaFree(p);
  };
  for (int d = 0; d < 3; ++d) {
    fr(s->tabs[d]);
    fr(s->dsym[d]);
  }
  fr(s->W1);
  fr(s->W2);
  if (!s->green_key.empty()) {
    std::lock_guard<std::mutex> lk(g_green_mu);
    auto it = g_green_cache.find(s->green_key);
    if (it != g_green_cache.end() && --it->second.refs == 0) {
      fr(it->second.dev);
      g_green_cache.erase(it);
    }
    s->green_dev = nullptr;
    s->green_key.clear();
  }
  fr(s->green_dev);
  fr(s->stage);
  fr(s->errflag);
  fr(s->gmaps_dev);
}

int flups_cleanup(flups_solver s) {
  if (!s) return FLUPS_OK;
  release(s, nullptr, false);
  delete s;
  return FLUPS_OK;
}

int flups_cleanup_async(flups_solver s, void* stream) {
  if (!s) return FLUPS_OK;
  release(s, (cudaStream_t)stream, true);
  delete s;
  return FLUPS_OK;
}

int flups_solver_share_green(flups_solver s) {
  if (!s) return FLUPS_EINVAL;
  if (s->ready) return FLUPS_ESTATE;
  s->share_green = true;
  return FLUPS_OK;
}

int flups_solver_check(flups_solver s, int* code) {
  if (!s || !code) return FLUPS_EINVAL;
  *code = 0;
  if (!s->errflag) return FLUPS_OK;
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(code, s->errflag, sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemset(s->errflag, 0, sizeof(int)));
  return FLUPS_OK;
}

int flups_solver_order(flups_solver s, int order[3]) {
  if (!s || !order) return FLUPS_EINVAL;
  for (int i = 0; i < 3; ++i) order[i] = s->order[i];
  return FLUPS_OK;
}

int flups_solver_info(flups_solver s, int* launches_per_solve, int order[3], double* model_bytes, double* green_bytes) {
  if (!s) return FLUPS_EINVAL;
  if (!s->ready) return FLUPS_ESTATE;
  if (launches_per_solve) *launches_per_solve = (int)s->passes.size();
  if (order)
    for (int i = 0; i < 3; ++i) order[i] = s->order[i];
  if (model_bytes) *model_bytes = s->model_bytes;
  if (green_bytes) *green_bytes = s->green_bytes;
  return FLUPS_OK;
}

int flups_debug_special(int which, const double* x, const double* y, double* out, int n, double eps) {
  if (!x || !y || !out || n < 0) return FLUPS_EINVAL;
  GreenSampleParams q{};
  gauss_legendre(GL_N, q.gl_x, q.gl_w);
  cudaError_t e = launch_special_eval(which, x, y, out, n, eps, q, 0);
  if (e) return cuda_fail(e, "special eval");
  CK(cudaDeviceSynchronize());
  return FLUPS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free solve.
//
// Some callers must not allocate device memory at all: a host application
// that hands the whole device to its own pool allocator and forbids any other
// allocation, or a latency-critical loop that cannot afford the implicit
// device synchronisation of cudaMalloc/cudaFree.  For them
// flups_solve_periodic_noalloc runs the fully periodic solve with its whole
// workspace (intermediate spectra, twiddle tables, wavenumber tables) carved
// out of one file-scope device array of fixed size; it calls no cudaMalloc,
// cudaFree or allocating library routine.  The array exists once per device
// that loads the library and is held until the process exits.
// ---------------------------------------------------------------------------
#define FLUPS_NOALLOC_SCRATCH_BYTES (48u * 1024u * 1024u)

static __device__ __align__(256) unsigned char g_noalloc_scratch[FLUPS_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Twiddles exp(-2 pi i m/(2P)) (m < 2P) and |w|^2 of the periodic modes g < N/2 + 1, in FP64.
__global__ void k_noalloc_tables(double2* tw, int P, double* w2, int gext, double wscale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 2 * P) {
    double s, c;
    sincospi((double)i / (double)P, &s, &c);
    tw[i] = make_double2(c, -s);
  }
  if (i < gext) {
    const double w = wscale * i;
    w2[i] = w * w;
  }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int flups_solve_periodic_noalloc(double* phi, const double* rhs, const int n[3], const double L[3],
                                            void* stream) {
  if (!phi || !rhs || !n || !L) return FLUPS_EINVAL;
  for (int d = 0; d < 3; ++d) {
    if (!is_2a3b(n[d]) || n[d] < 4 || n[d] > 4096) return FLUPS_ESIZE;
    if (!(L[d] > 0.0)) return FLUPS_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return FLUPS_EINVAL;
  void* base = nullptr;
  {
    // set-up once per device, with that device current: the device address of the array
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
      g_noalloc_addr[dev] = p;
    }
    base = g_noalloc_addr[dev];
  }
  {
    const int rc = ensure_smem_limits();
    if (rc) return rc;
  }

  // plan: x R2C, y C2C, z fused C2C with the closed-form spectral kernel -1/|k|^2
  DirPlan dir[3];
  for (int d = 0; d < 3; ++d) {
    DirPlan& dp = dir[d];
    dp.type = T_PER;
    dp.n_data = n[d];
    dp.N = n[d];
    dp.P = n[d];
    dp.gext = n[d] / 2 + 1;
    dp.h = L[d] / n[d];
    dp.L = L[d];
    dp.wscale = 2.0 * M_PI / L[d];
    dp.rp = radix_plan(dp.P);
  }
  dir[0].role = R_R2C;
  dir[0].nm = dir[0].P / 2 + 1;
  dir[1].role = R_C2C;
  dir[1].nm = dir[1].P;
  dir[2].role = R_C2C;
  dir[2].nm = dir[2].P;
  int dims0[3] = {n[0], n[1], n[2]};
  int dims1[3] = {dir[0].nm, n[1], n[2]};
  int dims2[3] = {dir[0].nm, dir[1].nm, n[2]};
  const size_t es = sizeof(double);
  const size_t w1 = align256((size_t)dims1[0] * dims1[1] * dims1[2] * 2 * es);
  const size_t w2 = align256((size_t)dims2[0] * dims2[1] * dims2[2] * 2 * es);
  size_t off = 0;
  unsigned char* b = (unsigned char*)base;
  void* W1 = b + off;
  off += w1;
  void* W2 = b + off;
  off += w2;
  double* tabs[3];
  for (int d = 0; d < 3; ++d) {
    dir[d].tw = b + off;
    off += align256((size_t)2 * dir[d].P * 2 * es);
    tabs[d] = (double*)(b + off);
    off += align256((size_t)dir[d].gext * es);
  }
  if (off > FLUPS_NOALLOC_SCRATCH_BYTES) return FLUPS_ESIZE;
  for (int d = 0; d < 3; ++d) {
    const int cnt = 2 * dir[d].P;
    k_noalloc_tables<<<(cnt + 127) / 128, 128, 0, st>>>((double2*)dir[d].tw, dir[d].P, tabs[d], dir[d].gext,
                                                        dir[d].wscale);
    CK(cudaGetLastError());
  }
  Launch Ls[5];
  for (int i = 0; i < 5; ++i) Ls[i] = Launch{};
  Ls[0].kind = K_FWD_REAL;
  fill_geom(Ls[0], dir[0], 0, dims0, dims1, FLUPS_F64, true, FLUPS_CELL, 1);
  Ls[0].p.in = rhs;
  Ls[0].p.out = W1;
  Ls[1].kind = K_FWD_C2C;
  fill_geom(Ls[1], dir[1], 1, dims1, dims2, FLUPS_F64, false, FLUPS_CELL, 1);
  Ls[1].p.in = W1;
  Ls[1].p.out = W2;
  Ls[2].kind = K_FUSED_C2C;
  fill_geom(Ls[2], dir[2], 2, dims2, dims2, FLUPS_F64, false, FLUPS_CELL, 1);
  Ls[2].p.in = W2;
  Ls[2].p.out = W2;
  {
    FusedGreen& g = Ls[2].p.g;
    g.stored = nullptr;
    for (int d = 0; d < 3; ++d) {
      g.tab[d] = tabs[d];
      g.gext[d] = dir[d].gext;
      g.fold[d] = dir[d].role == R_C2C ? dir[d].P : 0;
    }
    g.kernel = FLUPS_SPECTRAL;
    g.scale = 1.0 / ((double)dir[0].P * dir[1].P * dir[2].P);
    g.dims1 = dims2[1];
    g.dims2 = dims2[2];
  }
  Ls[3].kind = K_INV_C2C;
  fill_geom(Ls[3], dir[1], 1, dims2, dims1, FLUPS_F64, false, FLUPS_CELL, 1);
  Ls[3].p.in = W2;
  Ls[3].p.out = W1;
  Ls[4].kind = K_INV_REAL;
  fill_geom(Ls[4], dir[0], 0, dims1, dims0, FLUPS_F64, true, FLUPS_CELL, 1);
  Ls[4].p.in = W1;
  Ls[4].p.out = phi;
  for (int i = 0; i < 5; ++i) {
    if (Ls[i].smem > 227 * 1024 || Ls[i].nthr > 1024) return FLUPS_ESIZE;
    cudaError_t e = launch_pass(Ls[i].kind, FLUPS_F64, Ls[i].p, Ls[i].grid, Ls[i].nthr, Ls[i].smem, st);
    if (e) return cuda_fail(e, "noalloc pass launch");
  }
  return FLUPS_OK;
}
