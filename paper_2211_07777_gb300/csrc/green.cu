// Green's function spectrum generation, FP64 on the device.
//
// The solve needs G^ = FFT of the Green's function on the extended domain
// (Section 2.3.1: G sampled on the doubled domain and symmetrised about L;
// Section 2.3.2: evaluated on the padded domain of a semi-unbounded direction
// and cosine-transformed).  For a symmetrised G the doubled-domain DFT is a
// type-I DCT of the samples G(m h), m = 0..M, so every unbounded-like
// direction is handled by one node-centred even-even forward pass on FP64
// data.  Spectral directions enter through their wavenumber: with d_u
// unbounded directions and spectral wavevector k_s the regularised kernel is
//     G(k_s, r) = - int_{eps^2/2}^inf exp(-t |k_s|^2) (4 pi t)^(-d_u/2) exp(-r^2/(4t)) dt,
// a partial Fourier transform of the fully spectral HEJ2 kernel
// -exp(-|k|^2 eps^2/2)/|k|^2 (Section "Validation": kernels HEJ2..HEJ10,
// HEJ0, LGF2, CHAT2).  Closed forms:
//   d_u = 3: -erf(r/(sqrt2 eps))/(4 pi r),    G(0) = -1/((2 pi)^{3/2} eps)
//   d_u = 1: k > 0: -(1/4k)[e^{-k z} erfc((k eps^2 - z)/(sqrt2 eps)) + e^{k z} erfc((k eps^2 + z)/(sqrt2 eps))]
//            k = 0: (z/2) erf(z/(sqrt2 eps)) + eps/sqrt(2 pi) e^{-z^2/(2 eps^2)}
//   d_u = 2: k = 0: (1/2pi)[ln r + E1(r^2/(2 eps^2))/2],  G(0) = (ln(2 eps^2) - gamma)/(4 pi)
//            k > 0: composite Gauss-Legendre quadrature of the integral in s = ln(2t/eps^2)
// and the spectrally truncated HEJ0 kernel (cut-off pi/h, d_u = 3):
//   -Si(pi r/h)/(2 pi^2 r),  G(0) = -1/(2 pi h).
#include <cuda_runtime.h>
#include <math.h>

#include "green.cuh"

namespace flups {

#define PI_D 3.14159265358979323846264338327950288
#define EULER_D 0.57721566490153286060651209008240243

// E1(x) for x > 0: power series for x <= 1, continued fraction (modified
// Lentz) of exp(x) E1(x) = 1/(x+1- 1/(x+3- 4/(x+5- ...))) otherwise.
__device__ double expint_e1(double x) {
  if (x <= 1.0) {
    double sum = 0.0, term = 1.0;
    for (int k = 1; k < 40; ++k) {
      term *= -x / k;
      const double add = term / k;
      sum += add;
      if (fabs(add) < 1e-18 * fabs(sum)) break;
    }
    return -EULER_D - log(x) - sum;
  }
  const double tiny = 1e-300;
  double b = x + 1.0, c = 1.0 / tiny, d = 1.0 / b, h = d;
  for (int i = 1; i < 500; ++i) {
    const double a = -(double)i * i;
    b += 2.0;
    d = 1.0 / (a * d + b);
    c = b + a / c;
    const double del = c * d;
    h *= del;
    if (fabs(del - 1.0) < 1e-16) break;
  }
  return h * exp(-x);
}

// Si(x), x >= 0: series for x <= 4, otherwise pi/2 + Im E1(i x) through the
// complex continued fraction of E1(z) at z = i x, since E1(ix) = -Ci(x) + i(Si(x) - pi/2).
__device__ double sine_integral(double x) {
  if (x <= 4.0) {
    const double x2 = x * x;
    double term = x, sum = x;
    for (int k = 1; k < 60; ++k) {
      term *= -x2 / ((2.0 * k) * (2.0 * k + 1.0));
      const double add = term / (2.0 * k + 1.0);
      sum += add;
      if (fabs(add) < 1e-18 * fabs(sum)) break;
    }
    return sum;
  }
  // Lentz on the complex fraction 1/(z+1- 1/(z+3- 4/(z+5- ...))), z = i x
  double br = 1.0, bi = x;                 // b = z + 1
  double cr = 1e300, ci = 0.0;             // c = 1/tiny
  double den = br * br + bi * bi;
  double dr = br / den, di = -bi / den;    // d = 1/b
  double hr = dr, hi = di;
  for (int i = 1; i < 1000; ++i) {
    const double a = -(double)i * i;
    br += 2.0;
    // d = 1/(a d + b)
    double tr = a * dr + br, ti = a * di + bi;
    den = tr * tr + ti * ti;
    dr = tr / den;
    di = -ti / den;
    // c = b + a/c
    den = cr * cr + ci * ci;
    cr = br + a * cr / den;
    ci = bi - a * ci / den;
    const double delr = cr * dr - ci * di, deli = cr * di + ci * dr;
    const double nr = hr * delr - hi * deli, ni = hr * deli + hi * delr;
    hr = nr;
    hi = ni;
    if (fabs(delr - 1.0) + fabs(deli) < 1e-16) break;
  }
  // E1(ix) = exp(-ix) h
  double s, c;
  sincos(x, &s, &c);
  const double e1i = -s * hr + c * hi;     // Im(exp(-ix) h) = Im((c - i s)(hr + i hi))
  return 0.5 * PI_D + e1i;                 // Si = pi/2 + Im E1(ix)
}

__device__ double hej2_du3(double r, double eps) {
  if (r == 0.0) return -1.0 / (pow(2.0 * PI_D, 1.5) * eps);
  return -erf(r / (sqrt(2.0) * eps)) / (4.0 * PI_D * r);
}

__device__ double hej0_du3(double r, double h) {
  if (r == 0.0) return -1.0 / (2.0 * PI_D * h);
  return -sine_integral(PI_D * r / h) / (2.0 * PI_D * PI_D * r);
}

__device__ double hej2_du1(double k, double z, double eps) {
  z = fabs(z);
  const double s2 = sqrt(2.0);
  if (k == 0.0) return 0.5 * z * erf(z / (s2 * eps)) + eps / sqrt(2.0 * PI_D) * exp(-z * z / (2.0 * eps * eps));
  const double a = k * eps / s2, b = z / (s2 * eps);
  const double gauss = exp(-a * a - b * b);
  const double tplus = erfcx(a + b) * gauss;
  const double amb = a - b;
  const double tminus = amb >= 0.0 ? erfcx(amb) * gauss : exp(-k * z) * erfc(amb);
  return -(tminus + tplus) / (4.0 * k);
}

__device__ double hej2_du2(double k, double r, double eps, const GreenSampleParams& q) {
  if (k == 0.0) {
    if (r == 0.0) return (log(2.0 * eps * eps) - EULER_D) / (4.0 * PI_D);
    return (log(r) + 0.5 * expint_e1(r * r / (2.0 * eps * eps))) / (2.0 * PI_D);
  }
  // -(1/4pi) int_0^inf exp(-a e^s - b e^-s) ds over the range where the exponent is below 50
  const double a = 0.5 * k * k * eps * eps, b = r * r / (2.0 * eps * eps);
  double lo, hi;
  if (b > 0.0) {
    const double c = sqrt(a * b);
    if (2.0 * c > 50.0) return 0.0;
    const double sstar = 0.5 * log(b / a);
    const double del = acosh(25.0 / c);
    lo = fmax(0.0, sstar - del);
    hi = sstar + del;
    if (hi <= lo) return 0.0;
  } else {
    if (a >= 50.0) return 0.0;
    lo = 0.0;
    hi = log(50.0 / a);
  }
  // exp(-a e^s - b e^-s) is bounded by 1 in the strip |Im s| < pi/2, so Gauss-Legendre
  // panels of width 1 (Bernstein ellipse parameter ~6.4) converge like 6.4^-32 with 16 nodes.
  // At node j of the panel centred at m, e^s = e^m e^{w x_j/2}: the node factors are the same in
  // every panel of this sample, so each node costs one exponential (of the integrand) instead of
  // three -- these samples are most of the setup time of plans with two unbounded directions
  // The nodes come in pairs x_{N-1-j} = -x_j (to the Newton iteration's 1e-16), whose factors
  // are each other's inverses: 8 factors and their inverses serve all 16 nodes.
  const int npan = max(1, (int)ceil(hi - lo));
  const double w = (hi - lo) / npan;
  constexpr int H = GL_N / 2;
  double ef[H], efi[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    ef[j] = exp(0.5 * w * q.gl_x[j]);
    efi[j] = 1.0 / ef[j];
  }
  double acc = 0.0;
  for (int pn = 0; pn < npan; ++pn) {
    const double em = exp(lo + (pn + 0.5) * w), emi = 1.0 / em;
    const double am = a * em, bm = b * emi;
    double pacc = 0.0;
#pragma unroll
    for (int j = 0; j < H; ++j)
      pacc += q.gl_w[j] * exp(-am * ef[j] - bm * efi[j]) + q.gl_w[GL_N - 1 - j] * exp(-am * efi[j] - bm * ef[j]);
    acc += 0.5 * w * pacc;
  }
  return -acc / (4.0 * PI_D);
}

// Order 2m kernels (m >= 2) from the order-2 one: the spectral HEJ2m kernel is
// -int_a^inf t^{m-1} |k|^{2(m-1)} e^{-t|k|^2} dt/(m-1)!  (a = eps^2/2), and
// |k|^{2n} e^{-t|k|^2} = (-d/dt)^n e^{-t|k|^2}; over the unbounded directions
// e^{-t|k|^2} becomes the heat kernel H(t) = e^{-t k_s^2}(4 pi t)^{-d_u/2} e^{-r^2/(4t)}.
// m - 1 integrations by parts leave
//     G_2m = G_2 + sum_{j=1}^{m-1} (-1)^j a^j H^{(j-1)}(a) / j!.
// The derivatives of H come from its logarithmic derivative
//     Lg(t) = (ln H)' = -k_s^2 - (d_u/2)/t + (r^2/4)/t^2,
//     Lg^{(p)}(t) = (-1)^p [-(d_u/2) p! t^{-p-1} + (r^2/4)(p+1)! t^{-p-2}],  p >= 1,
// and H^{(n+1)} = sum_{i<=n} C(n, i) H^{(i)} Lg^{(n-i)}.
__device__ double hej_higher_order_terms(int m, double k, double r, int du, double eps) {
  const double a = 0.5 * eps * eps;
  const double b = 0.25 * r * r, half_du = 0.5 * du;
  double H[5], Lg[4];
  H[0] = exp(-a * k * k - b / a) * pow(4.0 * PI_D * a, -half_du);
  Lg[0] = -k * k - half_du / a + b / (a * a);
  double fact = 1.0, sgn = -1.0;
  for (int p = 1; p < 4; ++p) {
    fact *= p;  // p!
    Lg[p] = sgn * (-half_du * fact * pow(a, -p - 1) + b * fact * (p + 1) * pow(a, -p - 2));
    sgn = -sgn;
  }
  for (int n = 0; n + 1 < m - 1; ++n) {
    double acc = 0.0, binom = 1.0;
    for (int i = 0; i <= n; ++i) {
      acc += binom * H[i] * Lg[n - i];
      binom = binom * (n - i) / (i + 1);
    }
    H[n + 1] = acc;
  }
  double out = 0.0, aj = 1.0, jfact = 1.0;
  for (int j = 1; j < m; ++j) {
    aj *= a;
    jfact *= j;
    out += ((j & 1) ? -1.0 : 1.0) * aj * H[j - 1] / jfact;
  }
  return out;
}

// The kernel's value at spectral wavenumber k and distance r over the unbounded directions.
__device__ __forceinline__ double green_value(const GreenSampleParams& q, double k, double r) {
  double v;
  if (q.kernel == 1) v = hej0_du3(r, q.hmax);
  else if (q.du == 3) v = hej2_du3(r, q.eps);
  else if (q.du == 2) v = hej2_du2(k, r, q.eps, q);
  else v = hej2_du1(k, r, q.eps);
  if (q.kernel == 0 && q.hej_m > 1) v += hej_higher_order_terms(q.hej_m, k, r, q.du, q.eps);
  return v;
}

// Every direction unbounded-like with one spacing h: the kernel is radial and r^2 = h^2 m with
// m = i^2 + j^2 + k^2, so it is evaluated once per m <= mmax (a table) and gathered -- the padded
// domains of semi-unbounded directions would otherwise evaluate it at tens of millions of points.
__global__ void k_green_radial_table(double* __restrict__ t, long long mmax, GreenSampleParams q) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m <= mmax; m += (long long)gridDim.x * blockDim.x)
    t[m] = green_value(q, 0.0, q.h[0] * sqrt((double)m));
}

__global__ void k_green_radial_gather(double* __restrict__ g, const double* __restrict__ t, GreenSampleParams q) {
  const long long tot = (long long)q.gext[0] * q.gext[1] * q.gext[2];
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx % q.gext[0], rest = idx / q.gext[0];
    const long long j = rest % q.gext[1], k = rest / q.gext[1];
    g[idx] = t[i * i + j * j + k * k];
  }
}

__global__ void __launch_bounds__(256, 2) k_green_sample(double* __restrict__ g, GreenSampleParams q) {
  const long long tot = (long long)q.gext[0] * q.gext[1] * q.gext[2];
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    int gi[3];
    gi[0] = (int)(idx % q.gext[0]);
    const long long rest = idx / q.gext[0];
    gi[1] = (int)(rest % q.gext[1]);
    gi[2] = (int)(rest / q.gext[1]);
    double k2 = 0.0, r2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      if (q.unb[d]) {
        const double r = gi[d] * q.h[d];
        r2 += r * r;
      } else {
        const double w = q.wscale[d] * (gi[d] + q.wshift[d]);
        k2 += w * w;
      }
    }
    g[idx] = green_value(q, sqrt(k2), sqrt(r2));
  }
}

// ---------------------------------------------------------------------------
// Lattice Green's function of the 7-point Laplacian (LGF2, every direction
// unbounded-like), with a unit source 1/(h0 h1 h2):
//     G(n) = -(1/(h0 h1 h2)) int_0^inf prod_d e^{-2t/h_d^2} I_{n_d}(2t/h_d^2) dt
// (1/sigma = int_0^inf e^{-t sigma} dt applied to the lattice symbol, and the
// generating function of I_n).  With t = hmin^2 s and c_d = hmin^2/h_d^2 the
// integrand is prod_d E(n_d, 2 c_d s), E(n, x) = e^{-x} I_n(x).  The integral
// is a fixed quadrature sum_q w_q prod_d E(n_d, 2 c_d s_q) up to s = T, plus the
// termwise integral of the large-argument expansion beyond T; the per-direction
// tables E(n, 2 c_d s_q), n = 0..nmax, make every sample a short dot product.
// ---------------------------------------------------------------------------

// a_j(n) (2c)^{-j} of e^{-x} I_n(x) ~ (2 pi x)^{-1/2} sum_j (-1)^j a_j(n) x^{-j}, x = 2 c s, as powers of 1/s
__device__ __forceinline__ void lgf_series(int n, double c, int J, double* out) {
  const double mu = 4.0 * (double)n * n;
  double a = 1.0;
  out[0] = 1.0;
  for (int j = 1; j < J; ++j) {
    a *= -(mu - (2.0 * j - 1.0) * (2.0 * j - 1.0)) / (8.0 * j * 2.0 * c);
    out[j] = a;
  }
}

// Table row of node q: E(n, x), n = 0..nmax, x = 2 c s_q, stored at B[q (nmax + 1) + n].
__global__ void k_lgf_table(double* __restrict__ B, const double* __restrict__ sq, int Q, int nmax, double c) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  double* row = B + (size_t)q * (nmax + 1);
  const double x = 2.0 * c * sq[q];
  if (x < 1.0) {
    // power series e^{-x} sum_k (x/2)^{2k+n} / (k! (k+n)!)
    const double ex = exp(-x), y = 0.25 * x * x;
    double lead = 1.0;  // (x/2)^n / n!
    for (int n = 0; n <= nmax; ++n) {
      double sum = 0.0, term = 1.0;
      for (int k = 0; k < 40; ++k) {
        if (k > 0) term *= y / ((double)k * (k + n));
        sum += term;
        if (term < 1e-18 * sum) break;
      }
      row[n] = ex * lead * sum;
      lead *= 0.5 * x / (n + 1);
    }
    return;
  }
  if (x > 50.0 * ((double)nmax * nmax + 1.0) && x > 400.0) {
    // large argument: (2 pi x)^{-1/2} sum_j (-1)^j a_j(n) / x^j, terms shrink at least 100x each
    const double pre = rsqrt(2.0 * PI_D * x);
    for (int n = 0; n <= nmax; ++n) {
      const double mu = 4.0 * (double)n * n;
      double term = 1.0, sum = 1.0;
      for (int j = 1; j < 12; ++j) {
        term *= -(mu - (2.0 * j - 1.0) * (2.0 * j - 1.0)) / (8.0 * j * x);
        sum += term;
        if (fabs(term) < 1e-18 * fabs(sum)) break;
      }
      row[n] = pre * sum;
    }
    return;
  }
  // Miller's backward recurrence I_{n-1} = I_{n+1} + (2n/x) I_n from far above nmax (where
  // I_n(x)/I_0(x) ~ exp(-n^2/(2x)) is negligible), normalised by e^{-x}(I_0 + 2 sum_{n>=1} I_n) = 1
  const int ns = nmax + 24 + (int)(10.0 * sqrt(x));
  const double ix = 1.0 / x;
  double up = 0.0, cur = 1e-280, sum = 0.0;
  for (int n = ns; n >= 1; --n) {
    const double dn = up + 2.0 * n * ix * cur;  // I_{n-1}
    sum += 2.0 * cur;                             // I_n, n >= 1
    if (n <= nmax) row[n] = cur;
    up = cur;
    cur = dn;
    if (fabs(cur) > 1e250) {
      up *= 1e-250;
      cur *= 1e-250;
      sum *= 1e-250;
      for (int m = n; m <= nmax; ++m) row[m] *= 1e-250;
    }
  }
  sum += cur;
  row[0] = cur;
  const double inv = 1.0 / sum;
  for (int n = 0; n <= nmax; ++n) row[n] *= inv;
}

struct LgfParams {
  int gext[3];
  int nmax[3];
  const double* B[3];   // per-direction tables [Q][nmax + 1]
  const double* w;      // quadrature weights (ds)
  int Q;
  double T;             // quadrature end; the tail beyond is integrated termwise
  double c[3];          // hmin^2 / h_d^2
  double scale;         // -hmin^2 / (h0 h1 h2)
};

__global__ void k_lgf_sample(double* __restrict__ g, LgfParams p) {
  const long long tot = (long long)p.gext[0] * p.gext[1] * p.gext[2];
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % p.gext[0]);
    const long long rest = idx / p.gext[0];
    const int j = (int)(rest % p.gext[1]), k = (int)(rest / p.gext[1]);
    const double* b0 = p.B[0] + i;
    const double* b1 = p.B[1] + j;
    const double* b2 = p.B[2] + k;
    const int s0 = p.nmax[0] + 1, s1 = p.nmax[1] + 1, s2 = p.nmax[2] + 1;
    double acc = 0.0;
    for (int q = 0; q < p.Q; ++q) acc += p.w[q] * b0[(size_t)q * s0] * b1[(size_t)q * s1] * b2[(size_t)q * s2];
    // tail: prod_d (4 pi c_d s)^{-1/2} (sum_j A_dj s^{-j}) over s > T
    constexpr int J = 7;
    double a0[J], a1[J], a2[J], c01[J];
    lgf_series(i, p.c[0], J, a0);
    lgf_series(j, p.c[1], J, a1);
    lgf_series(k, p.c[2], J, a2);
    for (int m = 0; m < J; ++m) {
      c01[m] = 0.0;
      for (int l = 0; l <= m; ++l) c01[m] += a0[l] * a1[m - l];
    }
    double tail = 0.0, tp = rsqrt(p.T);
    for (int m = 0; m < J; ++m) {
      double cm = 0.0;
      for (int l = 0; l <= m; ++l) cm += c01[l] * a2[m - l];
      tail += cm * tp / (0.5 + m);
      tp /= p.T;
    }
    tail *= rsqrt(64.0 * PI_D * PI_D * PI_D * p.c[0] * p.c[1] * p.c[2]);
    g[idx] = p.scale * (acc + tail);
  }
}

cudaError_t launch_lgf(double* g, const int* gext, const double* h, cudaStream_t st) {
  // quadrature in s: one 32-node Gauss-Legendre panel on [0, 2], then 16-node panels of width 1/3 in ln s
  double x32[32], w32[32], x16[16], w16[16];
  host_gauss_legendre(32, x32, w32);
  host_gauss_legendre(16, x16, w16);
  const double hmin = fmin(h[0], fmin(h[1], h[2]));
  double c[3], T = 1e5;
  int nmax[3];
  for (int d = 0; d < 3; ++d) {
    c[d] = hmin * hmin / (h[d] * h[d]);
    nmax[d] = gext[d] - 1;
    T = fmax(T, 400.0 * ((double)nmax[d] * nmax[d] + 1.0) / c[d]);
  }
  const double u0 = log(2.0), u1 = log(T);
  const int npan = (int)ceil((u1 - u0) * 3.0);
  const double du = (u1 - u0) / npan;
  const int Q = 32 + 16 * npan;
  double* hs = (double*)malloc(2 * sizeof(double) * Q);
  if (!hs) return cudaErrorMemoryAllocation;
  double* hw = hs + Q;
  for (int i = 0; i < 32; ++i) {
    hs[i] = 1.0 + x32[i];
    hw[i] = w32[i];
  }
  for (int pn = 0; pn < npan; ++pn)
    for (int i = 0; i < 16; ++i) {
      const double u = u0 + du * (pn + 0.5 * (x16[i] + 1.0));
      const double sv = exp(u);
      hs[32 + 16 * pn + i] = sv;
      hw[32 + 16 * pn + i] = 0.5 * du * w16[i] * sv;
    }
  size_t tab = 0;
  for (int d = 0; d < 3; ++d) tab += (size_t)Q * (nmax[d] + 1);
  double* dev = nullptr;
  cudaError_t e = cudaMallocAsync(&dev, (2 * (size_t)Q + tab) * sizeof(double), st);
  if (e) { free(hs); return e; }
  e = cudaMemcpyAsync(dev, hs, 2 * sizeof(double) * Q, cudaMemcpyHostToDevice, st);
  if (!e) e = cudaStreamSynchronize(st);
  free(hs);
  LgfParams p{};
  double* t = dev + 2 * (size_t)Q;
  for (int d = 0; d < 3 && !e; ++d) {
    p.gext[d] = gext[d];
    p.nmax[d] = nmax[d];
    p.c[d] = c[d];
    p.B[d] = t;
    k_lgf_table<<<(Q + 63) / 64, 64, 0, st>>>(t, dev, Q, nmax[d], c[d]);
    e = cudaGetLastError();
    t += (size_t)Q * (nmax[d] + 1);
  }
  if (!e) {
    p.w = dev + Q;
    p.Q = Q;
    p.T = T;
    p.scale = -hmin * hmin / (h[0] * h[1] * h[2]);
    const long long tot = (long long)gext[0] * gext[1] * gext[2];
    long long blocks = (tot + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_lgf_sample<<<(unsigned)blocks, 256, 0, st>>>(g, p);
    e = cudaGetLastError();
  }
  cudaFreeAsync(dev, st);
  return e;
}

// Path-precision copy of the FP64 samples, x rows of gx values laid out with pitch gp >= gx.
template <typename T>
__global__ void k_green_finalize(const double* __restrict__ g, T* __restrict__ out, long long n, int gx, int gp,
                                 double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[(i / gx) * gp + i % gx] = (T)(g[i] * scale);
}

// double-float storage: hi = nearest float, lo = nearest float of the remainder
__global__ void k_green_finalize_df(const double* __restrict__ g, float2* __restrict__ out, long long n, int gx, int gp,
                                    double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = g[i] * scale;
    const float h = __double2float_rn(v);
    out[(i / gx) * gp + i % gx] = make_float2(h, __double2float_rn(v - (double)h));
  }
}

// Fully spectral kernels evaluated in FP64 (stored spectrum of the double-float path):
// tab[d][g] holds |w_d|^2, or the 7-point symbol for LGF2; G = scale * f(sum_d tab[d][g_d]).
__global__ void k_green_spectral(double* __restrict__ g, int gx, int gy, int gz, const double* __restrict__ t0,
                                 const double* __restrict__ t1, const double* __restrict__ t2, int kernel,
                                 double eps2h, double scale) {
  const long long tot = (long long)gx * gy * gz;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i0 = (int)(idx % gx);
    const long long rest = idx / gx;
    const int i1 = (int)(rest % gy), i2 = (int)(rest / gy);
    const double k2 = t0[i0] + t1[i1] + t2[i2];
    double v = 0.0;
    if (k2 > 0.0) {
      if (kernel == 0 || kernel == 100) {
        v = -1.0 / k2;
      } else {
        const int m = kernel / 2;
        const double s = k2 * eps2h;
        double acc = 1.0, term = 1.0;
        for (int j = 1; j < m; ++j) {
          term = term * s / j;
          acc += term;
        }
        v = -exp(-s) * acc / k2;
      }
    }
    g[idx] = v * scale;
  }
}

cudaError_t launch_green_sample(double* g, const GreenSampleParams& q, cudaStream_t st) {
  const long long tot = (long long)q.gext[0] * q.gext[1] * q.gext[2];
  long long blocks = (tot + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  const bool same_h = fabs(q.h[1] - q.h[0]) <= 1e-13 * q.h[0] && fabs(q.h[2] - q.h[0]) <= 1e-13 * q.h[0];
  if (q.du == 3 && same_h) {
    long long mmax = 0;
    for (int d = 0; d < 3; ++d) mmax += (long long)(q.gext[d] - 1) * (q.gext[d] - 1);
    if (mmax + 1 < tot) {
      double* t = nullptr;
      cudaError_t e = cudaMallocAsync(&t, (size_t)(mmax + 1) * sizeof(double), st);
      if (e == cudaSuccess) {
        long long tb = (mmax + 256) / 256;
        if (tb > 152 * 64) tb = 152 * 64;
        k_green_radial_table<<<(unsigned)tb, 256, 0, st>>>(t, mmax, q);
        k_green_radial_gather<<<(unsigned)blocks, 256, 0, st>>>(g, t, q);
        e = cudaGetLastError();
        const cudaError_t e2 = cudaFreeAsync(t, st);
        return e ? e : e2;
      }
      cudaGetLastError();  // no room for the table: evaluate every sample
    }
  }
  k_green_sample<<<(unsigned)blocks, 256, 0, st>>>(g, q);
  return cudaGetLastError();
}

cudaError_t launch_green_finalize(const double* g, void* out, int prec, long long n, int gx, int gp, double scale,
                                  cudaStream_t st) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (prec == 0) k_green_finalize<float><<<(unsigned)blocks, 256, 0, st>>>(g, (float*)out, n, gx, gp, scale);
  else if (prec == 2) k_green_finalize_df<<<(unsigned)blocks, 256, 0, st>>>(g, (float2*)out, n, gx, gp, scale);
  else k_green_finalize<double><<<(unsigned)blocks, 256, 0, st>>>(g, (double*)out, n, gx, gp, scale);
  return cudaGetLastError();
}

cudaError_t launch_green_spectral(double* g, const int* gext, const double* const* tabs, int kernel, double eps2h,
                                  double scale, cudaStream_t st) {
  const long long n = (long long)gext[0] * gext[1] * gext[2];
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_green_spectral<<<(unsigned)blocks, 256, 0, st>>>(g, gext[0], gext[1], gext[2], tabs[0], tabs[1], tabs[2], kernel,
                                                     eps2h, scale);
  return cudaGetLastError();
}

// Device-side special functions exposed for tests through a small evaluation kernel.
__global__ void k_special_eval(int which, const double* __restrict__ x, const double* __restrict__ y, double* out, int n,
                               double eps, GreenSampleParams q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  switch (which) {
    case 0: out[i] = expint_e1(x[i]); break;
    case 1: out[i] = sine_integral(x[i]); break;
    case 2: out[i] = hej2_du1(x[i], y[i], eps); break;
    case 3: out[i] = hej2_du2(x[i], y[i], eps, q); break;
    case 4: out[i] = hej2_du3(y[i], eps); break;
    default:
      // 10 d_u + m (m = 2..5): the order-2m correction terms with d_u unbounded directions
      if (which >= 12 && which <= 35 && which % 10 >= 2 && which % 10 <= 5)
        out[i] = hej_higher_order_terms(which % 10, x[i], y[i], which / 10, eps);
      else
        out[i] = 0.0;
      break;
  }
}

cudaError_t launch_special_eval(int which, const double* x, const double* y, double* out, int n, double eps,
                                const GreenSampleParams& q, cudaStream_t st) {
  k_special_eval<<<(n + 127) / 128, 128, 0, st>>>(which, x, y, out, n, eps, q);
  return cudaGetLastError();
}

}  // namespace flups
