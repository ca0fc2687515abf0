"""Green's functions of the oracle (plain FP64 NumPy/SciPy, test infrastructure).

This module is test infrastructure: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA path.

The paper solves lap(u) = f as u = G * f (Section "Methodology", eq. poisson)
and defers the kernel formulas to its references (Section "Validation").  The
readings used here, all pinned by the tests against the paper's printed
convergence tables and against independent quadrature:

* spectral (the singular kernel on fully spectral BCs):  G^ = -1/|k|^2, G^(0) = 0.
* HEJ2m, regularised of order 2m: G = G0 * zeta_eps with a Gaussian-based
  smoothing zeta whose transform is exp(-s) * sum_{j<m} s^j/j!,  s = |k|^2 eps^2/2,
  eps = alpha*h (alpha = 2 by default).
* LGF2 on spectral BCs: the inverse 7-point finite-difference symbol.
* HEJ2 with d_u unbounded directions and spectral wavevector k_s (heat-kernel
  form, a partial Fourier transform of the spectral HEJ2 kernel):

      G(k_s, r) = - int_{eps^2/2}^inf exp(-t |k_s|^2) (4 pi t)^(-d_u/2) exp(-r^2/(4t)) dt

  with the closed forms below for d_u = 3, for d_u = 1 and for k_s = 0.
* HEJ2m, m >= 2, with d_u unbounded directions: the spectral kernel
  -Gamma(m, s)/((m-1)! |k|^2), s = |k|^2 eps^2/2, equals
  -int_a^inf t^{m-1} |k|^{2(m-1)} e^{-t|k|^2} dt/(m-1)!  (a = eps^2/2), and
  |k|^{2n} e^{-t|k|^2} = (-d/dt)^n e^{-t|k|^2}.  The partial inverse transform
  over the unbounded directions turns e^{-t|k|^2} into the heat kernel
  h(t) = exp(-t |k_s|^2) (4 pi t)^(-d_u/2) exp(-r^2/(4t)); integrating by parts
  m - 1 times leaves the HEJ2 kernel plus boundary terms at t = a:

      G_2m(k_s, r) = G_2(k_s, r) + sum_{j=1}^{m-1} (-1)^j a^j h^(j-1)(a) / j!

  (the terms at t = inf vanish for k_s > 0 or d_u = 3).
* HEJ0 (fully unbounded, spectral truncation of the kernel at |k| = pi/h):
  G = -Si(pi r / h)/(2 pi^2 r),  G(0) = -1/(2 pi h).
* LGF2 with every direction unbounded: the lattice Green's function of the
  7-point Laplacian, as an integral of products of scaled modified Bessel
  functions (lgf_3d).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

SQRT2 = math.sqrt(2.0)
EULER_GAMMA = 0.57721566490153286060651209008240243


# ---------------------------------------------------------------------------
# Fully spectral kernels, functions of the wavevector (Section "Validation",
# symmetric and periodic case).  k2 = |k|^2; kdir = per-direction wavenumbers.
# ---------------------------------------------------------------------------
def spectral_kernel(name: str, k2: np.ndarray, eps: float, kdir=None, h=None) -> np.ndarray:
    """G^(k) for fully spectral boundary conditions; the k = 0 mode is 0 (zero mean)."""
    k2 = np.asarray(k2, dtype=np.float64)
    out = np.zeros_like(k2)
    nz = k2 > 0.0
    if name == "spectral":
        out[nz] = -1.0 / k2[nz]
        return out
    if name.startswith("hej") and name != "hej0":
        m = int(name[3:]) // 2
        s = k2[nz] * eps * eps / 2.0
        acc = np.zeros_like(s)
        term = np.ones_like(s)
        for j in range(m):
            if j > 0:
                term = term * s / j
            acc = acc + term
        out[nz] = -np.exp(-s) * acc / k2[nz]
        return out
    if name == "lgf2":
        # inverse of the 7-point Laplacian symbol: sum_d (2 - 2 cos(k_d h_d)) / h_d^2
        sym = np.zeros_like(k2)
        for kd, hd in zip(kdir, h):
            sym = sym + (2.0 - 2.0 * np.cos(kd * hd)) / (hd * hd)
        nzs = sym > 0.0
        out = np.zeros_like(sym)
        out[nzs] = -1.0 / sym[nzs]
        return out
    raise ValueError(f"kernel {name!r} has no fully spectral form in the oracle")


# ---------------------------------------------------------------------------
# Real-space and mixed HEJ2 kernels.
# ---------------------------------------------------------------------------
def hej2_3d(r: np.ndarray, eps: float) -> np.ndarray:
    """d_u = 3: -erf(r/(sqrt2 eps))/(4 pi r), and -1/((2 pi)^{3/2} eps) at r = 0."""
    r = np.asarray(r, dtype=np.float64)
    out = np.full_like(r, -1.0 / ((2.0 * math.pi) ** 1.5 * eps))
    nz = r > 0.0
    out[nz] = -special.erf(r[nz] / (SQRT2 * eps)) / (4.0 * math.pi * r[nz])
    return out


def hej0_3d(r: np.ndarray, h: float) -> np.ndarray:
    """Spectrally truncated kernel (cut-off pi/h): -Si(pi r/h)/(2 pi^2 r), -1/(2 pi h) at 0."""
    r = np.asarray(r, dtype=np.float64)
    out = np.full_like(r, -1.0 / (2.0 * math.pi * h))
    nz = r > 0.0
    si, _ = special.sici(math.pi * r[nz] / h)
    out[nz] = -si / (2.0 * math.pi ** 2 * r[nz])
    return out


def hej2_1d(k: np.ndarray, z: np.ndarray, eps: float) -> np.ndarray:
    """d_u = 1 (one unbounded direction, spectral wavenumber |k_s| = k).

    k > 0: -(1/4k)[e^{-k|z|} erfc((k eps^2 - |z|)/(sqrt2 eps)) + e^{k|z|} erfc((k eps^2 + |z|)/(sqrt2 eps))]
    k = 0: (|z|/2) erf(|z|/(sqrt2 eps)) + eps/sqrt(2 pi) exp(-z^2/(2 eps^2))   (1D Green |z|/2, smoothed)
    The k > 0 form is evaluated with erfcx so that no exponential overflows.
    """
    k, z = np.broadcast_arrays(np.asarray(k, dtype=np.float64), np.abs(np.asarray(z, dtype=np.float64)))
    out = np.empty(k.shape, dtype=np.float64)
    zero = k == 0.0
    zz = z[zero]
    out[zero] = 0.5 * zz * special.erf(zz / (SQRT2 * eps)) + eps / math.sqrt(2.0 * math.pi) * np.exp(-zz * zz / (2.0 * eps * eps))
    kk = k[~zero]
    zz = z[~zero]
    a = kk * eps / SQRT2
    b = zz / (SQRT2 * eps)
    gauss = np.exp(-a * a - b * b)
    # e^{k|z|} erfc(a + b) = erfcx(a + b) exp(-a^2 - b^2)
    t_plus = special.erfcx(a + b) * gauss
    # e^{-k|z|} erfc(a - b): erfcx form when a >= b, direct form otherwise (no overflow either way)
    amb = a - b
    t_minus = np.where(amb >= 0.0, special.erfcx(np.maximum(amb, 0.0)) * gauss,
                       np.exp(-kk * zz) * special.erfc(np.minimum(amb, 0.0)))
    out[~zero] = -(t_minus + t_plus) / (4.0 * kk)
    return out


def _gauss_legendre(n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


_GL_X, _GL_W = _gauss_legendre(24)


def hej2_2d(k: np.ndarray, r: np.ndarray, eps: float) -> np.ndarray:
    """d_u = 2 (two unbounded directions, spectral wavenumber |k_s| = k).

    k = 0: (1/2pi)[ln r + E1(r^2/(2 eps^2))/2], and (ln(2 eps^2) - gamma)/(4 pi) at r = 0.
    k > 0: the heat-kernel integral, with t = (eps^2/2) e^s:
        G = -(1/4pi) int_0^inf exp(-a e^s - b e^{-s}) ds,  a = k^2 eps^2/2,  b = r^2/(2 eps^2),
    by composite Gauss-Legendre on [0, s_max] where a e^{s_max} = 60.
    """
    k, r = np.broadcast_arrays(np.asarray(k, dtype=np.float64), np.asarray(r, dtype=np.float64))
    out = np.empty(k.shape, dtype=np.float64)
    zero = k == 0.0
    rz = r[zero]
    g0 = np.full(rz.shape, (math.log(2.0 * eps * eps) - EULER_GAMMA) / (4.0 * math.pi))
    nzr = rz > 0.0
    g0[nzr] = (np.log(rz[nzr]) + 0.5 * special.exp1(rz[nzr] ** 2 / (2.0 * eps * eps))) / (2.0 * math.pi)
    out[zero] = g0

    kk = k[~zero].ravel()
    rr = r[~zero].ravel()
    a = kk * kk * eps * eps / 2.0
    b = rr * rr / (2.0 * eps * eps)
    smax = np.log(np.maximum(60.0 / a, math.e))
    npan = np.maximum(np.ceil(smax / 0.25).astype(np.int64), 1)
    res = np.zeros_like(a)
    # integrate panel by panel; points with fewer panels simply stop contributing
    for p in range(int(npan.max()) if npan.size else 0):
        live = npan > p
        if not np.any(live):
            break
        width = smax[live] / npan[live]
        lo = p * width
        s = lo[:, None] + 0.5 * width[:, None] * (_GL_X[None, :] + 1.0)
        f = np.exp(-a[live, None] * np.exp(s) - b[live, None] * np.exp(-s))
        res[live] += 0.5 * width * (f @ _GL_W)
    out[~zero] = (-res / (4.0 * math.pi)).reshape(kk.shape) if kk.size else res
    return out


def hej2_mixed(du: int, kmag: np.ndarray, r: np.ndarray, eps: float) -> np.ndarray:
    """HEJ2 kernel with du unbounded directions, |k_s| = kmag and distance r."""
    if du == 3:
        return hej2_3d(r, eps)
    if du == 2:
        return hej2_2d(kmag, r, eps)
    if du == 1:
        return hej2_1d(kmag, r, eps)
    raise ValueError("du must be 1, 2 or 3 here")


# ---------------------------------------------------------------------------
# Higher-order regularised kernels (HEJ4 ... HEJ10) with unbounded directions.
# ---------------------------------------------------------------------------
def heat_kernel_derivatives(n: int, t: float, q: np.ndarray, du: int, b: np.ndarray):
    """[h^(0)(t), ..., h^(n)(t)] for h(t) = e^{-t q} (4 pi t)^(-du/2) e^{-b/t},
    by the general Leibniz rule over the three factors:
      (e^{-tq})^(i)        = (-q)^i e^{-tq}
      (t^{-du/2})^(i)      = prod_{l<i} (-du/2 - l) t^{-du/2-i}
      (e^{-b/t})^(i)       = e^{-b/t} P_i(1/t),  P_0 = 1,  P_{i+1} = P_i' + (b/t^2) P_i
    (P_i is kept as coefficients of powers of u = 1/t:  d/dt u^p = -p u^{p+1})."""
    q = np.asarray(q, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    u = 1.0 / t
    A = [(-q) ** i * np.exp(-t * q) for i in range(n + 1)]
    B = []
    for i in range(n + 1):
        c = 1.0
        for l in range(i):
            c *= -du / 2.0 - l
        B.append(c * (4.0 * math.pi) ** (-du / 2.0) * t ** (-du / 2.0 - i))
    polys = [{0: np.ones_like(b)}]
    for i in range(n):
        nxt = {}
        for pw, c in polys[-1].items():
            if pw > 0:
                nxt[pw + 1] = nxt.get(pw + 1, 0.0) - pw * c
            nxt[pw + 2] = nxt.get(pw + 2, 0.0) + b * c
        polys.append(nxt)
    eb = np.exp(-b * u)
    C = [eb * sum(c * u ** pw for pw, c in P.items()) for P in polys]
    out = []
    for m in range(n + 1):
        acc = 0.0
        for i in range(m + 1):
            for j in range(m - i + 1):
                l = m - i - j
                coef = math.factorial(m) // (math.factorial(i) * math.factorial(j) * math.factorial(l))
                acc = acc + coef * A[i] * B[j] * C[l]
        out.append(acc)
    return out


def hej_mixed(m: int, du: int, kmag: np.ndarray, r: np.ndarray, eps: float) -> np.ndarray:
    """HEJ2m kernel (order 2m) with du unbounded directions, |k_s| = kmag, distance r."""
    kmag, r = np.broadcast_arrays(np.asarray(kmag, dtype=np.float64), np.asarray(r, dtype=np.float64))
    g = hej2_mixed(du, kmag, r, eps)
    if m == 1:
        return g
    a = eps * eps / 2.0
    hd = heat_kernel_derivatives(m - 2, a, kmag * kmag, du, r * r / 4.0)
    for j in range(1, m):
        g = g + (-1.0) ** j * a ** j * hd[j - 1] / math.factorial(j)
    return g


# ---------------------------------------------------------------------------
# Lattice Green's function (LGF2) with every direction unbounded.
# ---------------------------------------------------------------------------
def _ive_series_coeffs(nu: np.ndarray, J: int):
    """a_j(nu), j < J, of the large-x expansion e^{-x} I_nu(x) ~ (2 pi x)^{-1/2} sum_j (-1)^j a_j / x^j,
    a_j = prod_{i=1..j} (4 nu^2 - (2i-1)^2) / (j! 8^j)."""
    mu = 4.0 * np.asarray(nu, dtype=np.float64) ** 2
    out = [np.ones_like(mu)]
    for j in range(1, J):
        out.append(out[-1] * (mu - (2 * j - 1) ** 2) / (j * 8.0))
    return out


def lgf_3d(n0, n1, n2, h) -> np.ndarray:
    """Lattice Green's function of the 7-point Laplacian sum_d (u(n+e_d) - 2u(n) + u(n-e_d))/h_d^2
    with a unit source 1/(h0 h1 h2) at the origin, at integer offsets (n0, n1, n2):

        G(n) = -(1/(h0 h1 h2)) int_0^inf prod_d e^{-2t/h_d^2} I_{n_d}(2t/h_d^2) dt

    (1/sigma(theta) = int_0^inf e^{-t sigma} dt and (1/2pi) int e^{i n theta} e^{2s cos theta} dtheta = I_n(2s)).
    Quadrature: t = hmin^2 s; Gauss-Legendre on s in [0, 1], on panels of width 1/4 in ln s up to T,
    and beyond T the large-argument expansion of each factor integrated term by term."""
    n = [np.abs(np.asarray(v, dtype=np.int64)) for v in (n0, n1, n2)]
    n = np.broadcast_arrays(*n)
    hmin = min(h)
    c = [hmin * hmin / (hd * hd) for hd in h]
    nmax = [int(v.max()) if v.size else 0 for v in n]
    T = max(1.0e4, max(100.0 * (nm * nm + 1) / cd for nm, cd in zip(nmax, c)))
    x16, w16 = np.polynomial.legendre.leggauss(16)
    nodes, weights = [], []
    for lo, hi in ((0.0, 0.5), (0.5, 1.0)):
        nodes.append(lo + (hi - lo) * (x16 + 1) / 2)
        weights.append((hi - lo) / 2 * w16)
    npan = int(math.ceil(math.log(T) / 0.25))
    du = math.log(T) / npan
    for p in range(npan):
        u = p * du + du * (x16 + 1) / 2
        s = np.exp(u)
        nodes.append(s)
        weights.append(du / 2 * w16 * s)
    s = np.concatenate(nodes)
    w = np.concatenate(weights)
    B = [special.ive(np.arange(nm + 1)[:, None], 2.0 * cd * s[None, :]) for nm, cd in zip(nmax, c)]
    flat = [v.ravel() for v in n]
    F = np.empty(flat[0].shape, dtype=np.float64)
    chunk = 4096
    for i in range(0, F.size, chunk):
        sl = slice(i, i + chunk)
        F[sl] = (B[0][flat[0][sl]] * B[1][flat[1][sl]] * B[2][flat[2][sl]]) @ w
    # tail: prod_d (4 pi c_d s)^{-1/2} sum_j (-1)^j a_j(n_d) (2 c_d s)^{-j}, integrated over s > T
    J = 6
    poly = np.ones((F.size, 1))
    for d in range(3):
        a = _ive_series_coeffs(flat[d], J)
        fac = np.stack([(-1.0) ** j * a[j] * (2.0 * c[d]) ** (-j) for j in range(J)], axis=1)
        prod = np.zeros((F.size, poly.shape[1] + J - 1))
        for j in range(J):
            prod[:, j:j + poly.shape[1]] += fac[:, j:j + 1] * poly
        poly = prod[:, :J]
    K = 1.0
    for cd in c:
        K /= math.sqrt(4.0 * math.pi * cd)
    tail = np.zeros(F.size)
    for j in range(J):
        tail += poly[:, j] * T ** (-0.5 - j) / (0.5 + j)
    F += K * tail
    return (-(hmin * hmin) / (h[0] * h[1] * h[2]) * F).reshape(n[0].shape)
