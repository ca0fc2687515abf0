"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here runs the CUDA path.  Each test pins a part of ``oracle/`` to
something other than itself: the paper's printed E_inf tables (golden
fixtures), the paper's transform definitions written as O(N^2) sums, adaptive
quadrature of the kernel integrals, O(N^6) direct convolutions and closed-form
potentials.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

import oracle
from oracle import CELL, NODE, EVEN, ODD, PER, UNB, Problem, solve
from oracle import green
from tests import analytic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_einf.json")


# ---------------------------------------------------------------------------
# 1. Extensions against the paper's transform definitions (Section 2.2).
# ---------------------------------------------------------------------------
def _dft(e):
    P = e.shape[0]
    j = np.arange(P)
    return np.exp(-2j * math.pi * np.outer(j, j) / P) @ e


def _node_defs(f):
    """The four node-centred r2r transforms of Section 2.2.1-2.2.4, as O(N^2) sums."""
    N = f.size - 1
    j = np.arange(1, N)
    k = np.arange(N + 1)
    dct1 = f[0] + (-1.0) ** k * f[N] + 2 * np.cos(math.pi * np.outer(k, j) / N) @ f[1:N]
    k1 = np.arange(1, N)
    dst1 = 2 * np.sin(math.pi * np.outer(k1, j) / N) @ f[1:N]
    m = np.arange(N)
    dst3 = (-1.0) ** m * f[N] + 2 * np.sin(math.pi * np.outer(m + 0.5, j) / N) @ f[1:N]
    dct3 = f[0] + 2 * np.cos(math.pi * np.outer(m + 0.5, j) / N) @ f[1:N]
    return dct1, dst1, dst3, dct3


def _cell_defs(f):
    """Textbook cell-centred transforms DCT-II, DST-II, DCT-IV, DST-IV (Table 1)."""
    N = f.size
    j = np.arange(N) + 0.5
    k = np.arange(N + 1)
    dct2 = 2 * np.cos(math.pi * np.outer(k, j) / N) @ f
    dst2 = 2 * np.sin(math.pi * np.outer(k, j) / N) @ f
    m = np.arange(N) + 0.5
    dct4 = 2 * np.cos(math.pi * np.outer(m, j) / N) @ f
    dst4 = 2 * np.sin(math.pi * np.outer(m, j) / N) @ f
    return dct2, dst2, dct4, dst4


@pytest.mark.parametrize("N", [7, 8, 12])
def test_node_extensions_match_paper_transforms(N):
    rng = np.random.default_rng(N)
    f = rng.standard_normal(N + 1)
    dct1, dst1, dst3, dct3 = _node_defs(f)
    E = _dft(oracle.extend(f, "EE", NODE))
    assert E.size == 2 * N
    np.testing.assert_allclose(E[:N + 1], dct1, atol=1e-12)
    E = _dft(oracle.extend(f, "OO", NODE))
    np.testing.assert_allclose(E[1:N], -1j * dst1, atol=1e-12)
    assert abs(E[0]) < 1e-12 and abs(E[N]) < 1e-12
    E = _dft(oracle.extend(f, "OE", NODE))
    assert E.size == 4 * N
    np.testing.assert_allclose(E[1:2 * N:2], -2j * dst3, atol=1e-12)
    np.testing.assert_allclose(E[0::2], 0, atol=1e-12)
    E = _dft(oracle.extend(f, "EO", NODE))
    np.testing.assert_allclose(E[1:2 * N:2], 2 * dct3, atol=1e-12)
    np.testing.assert_allclose(E[0::2], 0, atol=1e-12)
    # periodic: f_N unused, eq. of Section 2.2 (DFT of the N first samples)
    E = _dft(oracle.extend(f, "PER", NODE))
    jj = np.arange(N)
    np.testing.assert_allclose(E, np.exp(-2j * math.pi * np.outer(jj, jj) / N) @ f[:N], atol=1e-12)
    # unbounded: N+1 values then N-1 zeros (period 2N)
    e = oracle.extend(f, "UNB", NODE)
    assert e.size == 2 * N and np.all(e[N + 1:] == 0) and np.all(e[:N + 1] == f)


@pytest.mark.parametrize("N", [6, 8, 9])
def test_cell_extensions_match_textbook_transforms(N):
    rng = np.random.default_rng(100 + N)
    f = rng.standard_normal(N)
    dct2, dst2, dct4, dst4 = _cell_defs(f)
    k = np.arange(2 * N)
    shift2 = np.exp(-1j * math.pi * k / (2 * N))       # samples at (j + 1/2) h
    E = shift2 * _dft(oracle.extend(f, "EE", CELL))
    np.testing.assert_allclose(E[:N + 1], dct2, atol=1e-12)
    E = shift2 * _dft(oracle.extend(f, "OO", CELL))
    np.testing.assert_allclose(E[:N + 1], -1j * dst2, atol=1e-12)
    k4 = np.arange(4 * N)
    shift4 = np.exp(-1j * math.pi * k4 / (4 * N))
    E = shift4 * _dft(oracle.extend(f, "EO", CELL))
    np.testing.assert_allclose(E[1:2 * N:2], 2 * dct4, atol=1e-12)
    np.testing.assert_allclose(E[0::2], 0, atol=1e-12)
    E = shift4 * _dft(oracle.extend(f, "OE", CELL))
    np.testing.assert_allclose(E[1:2 * N:2], -2j * dst4, atol=1e-12)
    # scipy's DCT/DST (FFTW conventions) as a second, library statement of the same sums
    from scipy import fft as sfft
    np.testing.assert_allclose(dct2[:N], sfft.dct(f, type=2), atol=1e-12)
    np.testing.assert_allclose(dst2[1:], sfft.dst(f, type=2), atol=1e-12)
    np.testing.assert_allclose(dct4, sfft.dct(f, type=4), atol=1e-12)
    np.testing.assert_allclose(dst4, sfft.dst(f, type=4), atol=1e-12)


@pytest.mark.parametrize("center", [CELL, NODE])
def test_semi_unbounded_extensions(center):
    """Pad the unbounded side to 2L, then the symmetric transform on the padded domain (Section 2.3.2)."""
    N = 6
    rng = np.random.default_rng(7)
    n = N if center == CELL else N + 1
    f = rng.standard_normal(n)
    for t, refl in (("EU", "EE"), ("OU", "OO")):
        pad = np.concatenate([f, np.zeros(N)])
        np.testing.assert_array_equal(oracle.extend(f, t, center), oracle.extend(pad, refl, center))
        # unbounded on the left: the same on the reversed samples
        np.testing.assert_array_equal(oracle.extend(f, t[::-1], center), oracle.extend(f[::-1], t, center))
        assert oracle.extend(f, t, center).size == 4 * N


@pytest.mark.parametrize("center", [CELL, NODE])
@pytest.mark.parametrize("t", ["PER", "UNB", "EE", "EO", "OE", "OO", "EU", "OU", "UE", "UO"])
def test_restrict_inverts_extend(center, t):
    N = 8
    n = N if center == CELL else N + 1
    f = np.random.default_rng(3).standard_normal(n)
    g = oracle.restrict(oracle.extend(f, t, center), n, t, center)
    want = f.copy()
    if center == NODE:
        if t == "PER":
            want[N] = want[0]
        if t[0] == "O":
            want[0] = 0.0
        if t[1] == "O":
            want[N] = 0.0
    np.testing.assert_allclose(g, want, atol=0)


# ---------------------------------------------------------------------------
# 2. The paper's printed E_inf (golden fixtures).
# ---------------------------------------------------------------------------
with open(GOLDEN) as fh:
    _G = json.load(fh)


def _check_printed(err, printed):
    if printed < 1e-13:
        assert err < 5e-15, (err, printed)
    elif printed < 1e-10:
        assert abs(err - printed) < 1e-4 * printed + 1e-16, (err, printed)
    elif printed < 1e-6:
        assert abs(err - printed) < 1e-7 * printed, (err, printed)
    else:
        assert abs(err - printed) < 1e-10 * printed, (err, printed)


@pytest.mark.parametrize("npts", ["33", "65"])
@pytest.mark.parametrize("kernel", ["spectral", "lgf2", "hej2", "hej4", "hej6", "hej8", "hej10"])
def test_printed_symmetric_periodic(kernel, npts):
    N = int(npts) - 1
    phi, f = analytic.case_symmetric_periodic(N)
    h = 1.0 / N
    p = Problem(bc=((EVEN, EVEN), (ODD, EVEN), (PER, PER)), h=(h, h, h), center=NODE, kernel=kernel)
    err = np.abs(solve(f, p) - phi).max()
    _check_printed(err, _G["symmetric_periodic"][kernel][npts])


@pytest.mark.parametrize("npts", ["33", "65"])
@pytest.mark.parametrize("kernel", ["lgf2", "hej2", "hej4", "hej6", "hej8", "hej10", "hej0"])
def test_printed_unbounded(kernel, npts):
    N = int(npts) - 1
    phi, f = analytic.case_unbounded(N)
    h = 1.0 / N
    p = Problem(bc=((UNB, UNB),) * 3, h=(h, h, h), center=NODE, kernel=kernel)
    err = np.abs(solve(f, p) - phi).max()
    _check_printed(err, _G["unbounded"][kernel][npts])


@pytest.mark.parametrize("npts", ["33", "65"])
@pytest.mark.parametrize("kernel", ["lgf2", "hej2", "hej4", "hej6", "hej8", "hej10", "hej0"])
def test_printed_semi_unbounded(kernel, npts):
    N = int(npts) - 1
    phi, f = analytic.case_semi_unbounded(N)
    h = 1.0 / N
    p = Problem(bc=((UNB, EVEN), (UNB, UNB), (ODD, UNB)), h=(h, h, h), center=NODE, kernel=kernel)
    err = np.abs(solve(f, p) - phi).max()
    _check_printed(err, _G["semi_unbounded"][kernel][npts])


@pytest.mark.parametrize("case,kernel", [("unbounded", "hej4"), ("semi_unbounded", "hej2")])
def test_printed_at_129_points(case, kernel):
    """One kernel of each validation case at the next printed resolution (N + 1 = 129)."""
    N = 128
    h = 1.0 / N
    if case == "unbounded":
        phi, f = analytic.case_unbounded(N)
        bc = ((UNB, UNB),) * 3
    else:
        phi, f = analytic.case_semi_unbounded(N)
        bc = ((UNB, EVEN), (UNB, UNB), (ODD, UNB))
    err = np.abs(solve(f, Problem(bc=bc, h=(h, h, h), center=NODE, kernel=kernel)) - phi).max()
    _check_printed(err, _G[case][kernel]["129"])


# ---------------------------------------------------------------------------
# 3. Kernels against quadrature of their integral definitions.
# ---------------------------------------------------------------------------
EPS = 0.05


def _quad(du, k, r):
    fn = lambda t: math.exp(-t * k * k - r * r / (4 * t)) * (4 * math.pi * t) ** (-du / 2)
    v, _ = integrate.quad(fn, EPS * EPS / 2, np.inf, limit=500, epsabs=0, epsrel=1e-13)
    return -v


@pytest.mark.parametrize("k,z", [(1.0, 0.0), (3.0, 0.2), (50.0, 0.7), (0.01, 0.3), (20.0, 0.0)])
def test_hej2_1d_against_quadrature(k, z):
    g = green.hej2_1d(np.array([k]), np.array([z]), EPS)[0]
    q = _quad(1, k, z)
    assert abs(g - q) <= 1e-12 * abs(q) + 1e-300


def test_hej2_1d_large_argument_is_finite():
    g = green.hej2_1d(np.array([400.0, 4000.0]), np.array([0.9, 1.0]), EPS)
    assert np.all(np.isfinite(g)) and np.all(np.abs(g) < 1e-100)


def test_hej2_1d_zero_mode_is_finite_part_of_the_limit():
    """G(0, z) = lim_{k->0} [G(k, z) + 1/(2k)]: the constant is the finite part."""
    for z in (0.0, 0.1, 0.5):
        k = 1e-5
        lim = green.hej2_1d(np.array([k]), np.array([z]), EPS)[0] + 1 / (2 * k)
        g0 = green.hej2_1d(np.array([0.0]), np.array([z]), EPS)[0]
        assert abs(lim - g0) < 1e-4
    # far field of the smoothed |z|/2
    g0 = green.hej2_1d(np.array([0.0]), np.array([2.0]), EPS)[0]
    assert abs(g0 - 1.0) < 1e-14
    # second derivative = unit Gaussian of width eps
    z, d = 0.03, 1e-4
    gp = green.hej2_1d(np.zeros(3), np.array([z - d, z, z + d]), EPS)
    lap = (gp[0] - 2 * gp[1] + gp[2]) / d ** 2
    assert abs(lap - math.exp(-z * z / (2 * EPS ** 2)) / math.sqrt(2 * math.pi * EPS ** 2)) < 1e-5


@pytest.mark.parametrize("k,r", [(1.0, 0.0), (3.0, 0.2), (50.0, 0.7), (10.0, 0.01), (0.5, 0.9), (200.0, 0.05)])
def test_hej2_2d_against_quadrature(k, r):
    g = green.hej2_2d(np.array([k]), np.array([r]), EPS)[0]
    q = _quad(2, k, r)
    assert abs(g - q) <= 1e-12 * abs(q) + 1e-300


def test_hej2_2d_far_field_and_zero_mode():
    k, r = 2.0, 0.6
    g = green.hej2_2d(np.array([k]), np.array([r]), EPS)[0]
    assert abs(g + special.k0(k * r) / (2 * math.pi)) < 1e-13
    for r in (0.0, 0.3):
        kk = 1e-6
        lim = green.hej2_2d(np.array([kk]), np.array([r]), EPS)[0] - (math.log(kk / 2) + np.euler_gamma) / (2 * math.pi)
        g0 = green.hej2_2d(np.array([0.0]), np.array([r]), EPS)[0]
        assert abs(lim - g0) < 1e-7
    g0 = green.hej2_2d(np.array([0.0]), np.array([1.5]), EPS)[0]
    assert abs(g0 - math.log(1.5) / (2 * math.pi)) < 1e-14


def _spectral_hej(m, k):
    """The fully spectral HEJ2m kernel -exp(-s) sum_{j<m} s^j/j! / k^2, s = k^2 eps^2/2 (its definition)."""
    s = k * k * EPS * EPS / 2
    acc, term = 0.0, 1.0
    for j in range(m):
        if j > 0:
            term *= s / j
        acc += term
    return -math.exp(-s) * acc / (k * k)


@pytest.mark.parametrize("m", [2, 3, 4, 5])
@pytest.mark.parametrize("r", [0.0, 0.004, 0.05, 0.1, 0.3, 0.9])
def test_hej_higher_order_3d_against_inverse_transform(m, r):
    """d_u = 3: G(r) = (1/(2 pi^2 r)) int_0^inf G^(k) k sin(k r) dk (radial inverse Fourier transform
    of the spectral definition); at r = 0 the integrand is G^(k) k^2 / (2 pi^2)."""
    if r == 0.0:
        fn = lambda k: _spectral_hej(m, k) * k * k / (2 * math.pi ** 2)
    else:
        fn = lambda k: _spectral_hej(m, k) * k * math.sin(k * r) / (2 * math.pi ** 2 * r)
    q, _ = integrate.quad(fn, 0.0, 60.0 / EPS, limit=4000, epsabs=0, epsrel=1e-13)
    g = green.hej_mixed(m, 3, np.array([0.0]), np.array([r]), EPS)[0]
    assert abs(g - q) <= 1e-12 * abs(q)


@pytest.mark.parametrize("m", [2, 3, 5])
@pytest.mark.parametrize("k,z", [(1.0, 0.0), (3.0, 0.2), (30.0, 0.05), (0.5, 0.7)])
def test_hej_higher_order_1d_against_inverse_transform(m, k, z):
    """d_u = 1: G(k_s, z) = (1/pi) int_0^inf G^(sqrt(k_s^2 + w^2)) cos(w z) dw."""
    fn = lambda w: _spectral_hej(m, math.sqrt(k * k + w * w)) * math.cos(w * z) / math.pi
    q, _ = integrate.quad(fn, 0.0, 60.0 / EPS, limit=4000, epsabs=0, epsrel=1e-13)
    g = green.hej_mixed(m, 1, np.array([k]), np.array([z]), EPS)[0]
    assert abs(g - q) <= 1e-11 * abs(q)


@pytest.mark.parametrize("m", [2, 4, 5])
@pytest.mark.parametrize("k,r", [(1.0, 0.0), (3.0, 0.2), (30.0, 0.05), (0.5, 0.7)])
def test_hej_higher_order_2d_against_inverse_transform(m, k, r):
    """d_u = 2: G(k_s, r) = (1/(2 pi)) int_0^inf G^(sqrt(k_s^2 + w^2)) J0(w r) w dw."""
    fn = lambda w: _spectral_hej(m, math.sqrt(k * k + w * w)) * special.j0(w * r) * w / (2 * math.pi)
    q, _ = integrate.quad(fn, 0.0, 60.0 / EPS, limit=4000, epsabs=0, epsrel=1e-13)
    g = green.hej_mixed(m, 2, np.array([k]), np.array([r]), EPS)[0]
    assert abs(g - q) <= 1e-11 * abs(q)


def test_hej_higher_order_reduces_to_hej2():
    k = np.array([0.0, 2.0, 7.0])
    r = np.array([0.1, 0.0, 0.3])
    for du in (1, 2, 3):
        kk = np.zeros(3) if du == 3 else k
        assert np.array_equal(green.hej_mixed(1, du, kk, r, EPS), green.hej2_mixed(du, kk, r, EPS))


def test_lattice_green_origin_is_watson_constant():
    """G(0) h = -W/6 with Watson's simple-cubic integral W = (1/pi^3) int_[0,pi]^3 dtheta/(1 - sum cos/3)
    in its closed form sqrt(6)/(32 pi^3) Gamma(1/24) Gamma(5/24) Gamma(7/24) Gamma(11/24) (Glasser and
    Zucker): 1/sum_d (2 - 2 cos theta_d) = 1/(6 (1 - sum cos/3))."""
    W = math.sqrt(6) / (32 * math.pi ** 3) * math.gamma(1 / 24) * math.gamma(5 / 24) * math.gamma(7 / 24) \
        * math.gamma(11 / 24)
    for h in (1.0, 0.25):
        g0 = green.lgf_3d(np.array([0]), np.array([0]), np.array([0]), (h, h, h))[0]
        assert abs(g0 * h + W / 6) < 1e-15


@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (1.0, 0.7, 1.3)])
def test_lattice_green_is_discrete_fundamental_solution(h):
    """The 7-point Laplacian of G is 1/(h0 h1 h2) at the origin and 0 everywhere else."""
    n = 10
    i = np.arange(-n, n + 1)
    Z, Y, X = np.meshgrid(i, i, i, indexing="ij")
    G = green.lgf_3d(X, Y, Z, h)
    c = G[1:-1, 1:-1, 1:-1]
    lap = (G[1:-1, 1:-1, 2:] + G[1:-1, 1:-1, :-2] - 2 * c) / h[0] ** 2 \
        + (G[1:-1, 2:, 1:-1] + G[1:-1, :-2, 1:-1] - 2 * c) / h[1] ** 2 \
        + (G[2:, 1:-1, 1:-1] + G[:-2, 1:-1, 1:-1] - 2 * c) / h[2] ** 2
    vol = h[0] * h[1] * h[2]
    m = n - 1
    assert abs(lap[m, m, m] * vol - 1.0) < 1e-13
    lap[m, m, m] = 0.0
    assert np.abs(lap).max() * vol < 1e-13


@pytest.mark.parametrize("n", [(0, 0, 5), (10, 3, 2), (32, 32, 32), (64, 0, 1)])
def test_lattice_green_against_adaptive_quadrature(n):
    """The defining integral -int_0^inf prod_d e^{-2t} I_{n_d}(2t) dt by adaptive quadrature up to
    10^6 plus the termwise tail, independent of the oracle's fixed-node rule."""
    fn = lambda t: special.ive(n[0], 2 * t) * special.ive(n[1], 2 * t) * special.ive(n[2], 2 * t)
    pts = [0, 0.5, 1, 3, 10, 30, 100, 300, 1e3, 3e3, 1e4, 3e4, 1e5, 3e5, 1e6]
    q = sum(integrate.quad(fn, a, b, limit=400, epsabs=0, epsrel=1e-13)[0] for a, b in zip(pts[:-1], pts[1:]))
    # beyond T = 10^6: product of the three large-x series of e^{-x} I_k(x), x = 2t, integrated termwise
    ser = []
    for k in n:
        c, term = [1.0], 1.0
        for j in range(1, 6):
            term *= -(4 * k * k - (2 * j - 1) ** 2) / (8 * j)
            c.append(term)
        ser.append(np.array(c))
    prod = np.convolve(np.convolve(ser[0], ser[1]), ser[2])[:6]
    T = 1e6
    q += (4 * math.pi) ** -1.5 * sum(cj * 2.0 ** -j * T ** (-0.5 - j) / (0.5 + j) for j, cj in enumerate(prod))
    g = green.lgf_3d(np.array([n[0]]), np.array([n[1]]), np.array([n[2]]), (1.0, 1.0, 1.0))[0]
    assert abs(g + q) < 1e-12 * q


def test_lattice_green_far_field():
    """|n| -> inf: G -> -1/(4 pi |n| h) (the continuous fundamental solution)."""
    g = green.lgf_3d(np.array([200]), np.array([0]), np.array([0]), (1.0, 1.0, 1.0))[0]
    assert abs(g * 4 * math.pi * 200 + 1) < 1e-5


def test_hej2_3d_and_hej0_limits():
    assert abs(green.hej2_3d(np.array([1.0]), EPS)[0] + 1 / (4 * math.pi)) < 1e-15
    r = np.array([1e-9])
    assert abs(green.hej2_3d(r, EPS)[0] - green.hej2_3d(np.array([0.0]), EPS)[0]) < 1e-12
    q = _quad(3, 0.0, 0.07)
    assert abs(green.hej2_3d(np.array([0.07]), EPS)[0] - q) < 1e-13 * abs(q)
    h = 0.01
    assert abs(green.hej0_3d(np.array([1e-9]), h)[0] - green.hej0_3d(np.array([0.0]), h)[0]) < 1e-9
    # far field: Si -> pi/2 on average
    rr = np.linspace(5.0, 6.0, 2001)
    assert abs(np.mean(green.hej0_3d(rr, h) * 4 * math.pi * rr) + 1) < 1e-3


# ---------------------------------------------------------------------------
# 4. Direct sums: the definition of the unbounded and mixed solves.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("center", [CELL, NODE])
def test_unbounded_equals_direct_convolution(center):
    N = 6
    n = N if center == CELL else N + 1
    h = 1.0 / N
    rng = np.random.default_rng(11)
    f = rng.standard_normal((n, n, n))
    eps = 2 * h
    pos = (np.arange(n) + (0.5 if center == CELL else 0.0)) * h
    Z, Y, X = np.meshgrid(pos, pos, pos, indexing="ij")
    P = np.stack([Z.ravel(), Y.ravel(), X.ravel()], 1)
    d = np.sqrt(((P[:, None, :] - P[None, :, :]) ** 2).sum(-1))
    # G by quadrature (independent of the closed form), for distinct distances
    du, inv = np.unique(np.round(d, 12), return_inverse=True)
    gq = np.array([_quad_eps(3, 0.0, x, eps) for x in du])
    ref = (h ** 3 * gq[inv].reshape(d.shape) @ f.ravel()).reshape(f.shape)
    out = solve(f, Problem(bc=((UNB, UNB),) * 3, h=(h, h, h), center=center, kernel="hej2"))
    np.testing.assert_allclose(out, ref, atol=1e-12 * np.abs(ref).max())


def _quad_eps(du, k, r, eps):
    fn = lambda t: math.exp(-t * k * k - r * r / (4 * t)) * (4 * math.pi * t) ** (-du / 2)
    v, _ = integrate.quad(fn, eps * eps / 2, np.inf, limit=500, epsabs=0, epsrel=1e-13)
    return -v


@pytest.mark.parametrize("center", [CELL, NODE])
@pytest.mark.parametrize("ztype", ["UNB", "EU", "OU", "UE"])
def test_mixed_one_unbounded_direction_mode_by_mode(center, ztype):
    """f = cos(pi p x) sin(2 pi q y) g(z): phi = mode x (1D convolution of g with G(k_s, .))
    by images for the semi-unbounded directions."""
    N = 8
    n = N if center == CELL else N + 1
    h = 1.0 / N
    eps = 2 * h
    pos = (np.arange(n) + (0.5 if center == CELL else 0.0)) * h
    p, q = 2, 1
    kap = math.hypot(math.pi * p, 2 * math.pi * q)
    g = np.random.default_rng(5).standard_normal(n)
    zbc = {"UNB": (UNB, UNB), "EU": (EVEN, UNB), "OU": (ODD, UNB), "UE": (UNB, EVEN)}[ztype]
    if center == NODE and zbc[0] == ODD:
        g[0] = 0.0
    ypos = pos if center == CELL else np.arange(N) * h        # y periodic, node layout without f_N
    ny = ypos.size
    mode_x = np.cos(math.pi * p * pos)
    mode_y = np.sin(2 * math.pi * q * ypos)
    if center == NODE:
        mode_y = np.sin(2 * math.pi * q * pos)                 # stored with the duplicate node
        ny = n
    f = g[:, None, None] * mode_y[None, :, None] * mode_x[None, None, :]
    G = lambda r: _quad_eps(1, kap, abs(r), eps)
    conv = np.zeros(n)
    for i in range(n):
        for j in range(n):
            zi, zj = pos[i], pos[j]
            if ztype == "UNB":
                conv[i] += h * G(zi - zj) * g[j]
            elif ztype in ("EU", "OU"):
                # a node on the mirror plane is its own image: counted once
                s = 1.0 if ztype == "EU" else -1.0
                img = 0.0 if (center == NODE and j == 0) else s * G(zi + zj)
                conv[i] += h * (G(zi - zj) + img) * g[j]
            else:  # UE: images about z = L
                img = 0.0 if (center == NODE and j == N) else G(zi + zj - 2.0)
                conv[i] += h * (G(zi - zj) + img) * g[j]
    ref = conv[:, None, None] * mode_y[None, :, None] * mode_x[None, None, :]
    out = solve(f, Problem(bc=((EVEN, EVEN), (PER, PER), zbc), h=(h, h, h), center=center, kernel="hej2"))
    np.testing.assert_allclose(out, ref, atol=1e-11 * np.abs(ref).max())


def test_mixed_two_unbounded_directions_mode_by_mode():
    N = 6
    h = 1.0 / N
    eps = 2 * h
    pos = (np.arange(N) + 0.5) * h
    q = 1
    kap = 2 * math.pi * q
    g = np.random.default_rng(9).standard_normal((N, N))     # [z, y]
    mode_x = np.sin(2 * math.pi * q * pos)
    f = g[:, :, None] * mode_x[None, None, :]
    Zg, Yg = np.meshgrid(pos, pos, indexing="ij")
    conv = np.zeros((N, N))
    cache = {}
    for i in range(N):
        for j in range(N):
            r = np.sqrt((Zg[i, j] - Zg) ** 2 + (Yg[i, j] - Yg) ** 2)
            vals = np.zeros_like(r)
            for idx, rv in np.ndenumerate(r):
                key = round(rv, 12)
                if key not in cache:
                    cache[key] = _quad_eps(2, kap, rv, eps)
                vals[idx] = cache[key]
            conv[i, j] = h * h * (vals * g).sum()
    ref = conv[:, :, None] * mode_x[None, None, :]
    out = solve(f, Problem(bc=((PER, PER), (UNB, UNB), (UNB, UNB)), h=(h, h, h), center=CELL, kernel="hej2"))
    np.testing.assert_allclose(out, ref, atol=1e-11 * np.abs(ref).max())


# ---------------------------------------------------------------------------
# 5. Closed forms.
# ---------------------------------------------------------------------------
def test_periodic_sine_product_is_exact():
    from paper_2211_07777_gb300 import workloads as W
    modes = W.sine_modes(1)
    n = (32, 32, 32)
    f = W.periodic_sines(n, modes)
    phi = np.zeros_like(f)
    x = W.coords(32, 1.0, CELL)
    for a, b, c, A in modes:
        k2 = (2 * math.pi) ** 2 * (a * a + b * b + c * c)
        phi += -A / k2 * np.sin(2 * math.pi * c * x)[:, None, None] * np.sin(2 * math.pi * b * x)[None, :, None] \
            * np.sin(2 * math.pi * a * x)[None, None, :]
    h = 1 / 32
    out = solve(f, Problem(bc=((PER, PER),) * 3, h=(h, h, h), center=CELL, kernel="spectral"))
    assert np.abs(out - phi).max() < 1e-15 * 100


def test_gaussian_blob_regularised_closed_form():
    """With HEJ2 (Gaussian smoothing eps) the solve of a sigma-Gaussian is the potential of a
    Gaussian of width sqrt(sigma^2 + eps^2), up to the blob's truncation at the box."""
    from paper_2211_07777_gb300 import workloads as W
    N = 64
    h = 1.0 / N
    c = (0.5, 0.5, 0.5)
    f = W.gaussian_blob((N, N, N), 0.1, c)
    out = solve(f, Problem(bc=((UNB, UNB),) * 3, h=(h, h, h), center=CELL, kernel="hej2"))
    x = W.coords(N, 1.0, CELL) - 0.5
    r = np.sqrt(x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2)
    ref = analytic.gaussian_potential(r, math.sqrt(0.01 + (2 * h) ** 2))
    assert np.abs(out - ref).max() / np.abs(ref).max() < 1e-6


def test_biot_savart_periodic_closed_form():
    """lap(u) = curl(f) with f_x = sin(2 pi y) sin(4 pi z), f_y = cos(2 pi x) sin(2 pi z),
    f_z = sin(4 pi x) cos(2 pi y) on a periodic box: each curl term is an eigenfunction."""
    N = 16
    h = 1.0 / N
    x = (np.arange(N) + 0.5) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    tp = 2 * math.pi
    f = np.stack([np.sin(tp * Y) * np.sin(2 * tp * Z), np.cos(tp * X) * np.sin(tp * Z), np.sin(2 * tp * X) * np.cos(tp * Y)])
    # curl f, term by term, and the eigenvalue -|k|^2 of each term
    terms_x = [(-tp * np.sin(2 * tp * X) * np.sin(tp * Y), 4 + 1), (-tp * np.cos(tp * X) * np.cos(tp * Z), 1 + 1)]
    terms_y = [(2 * tp * np.sin(tp * Y) * np.cos(2 * tp * Z), 1 + 4), (-2 * tp * np.cos(2 * tp * X) * np.cos(tp * Y), 4 + 1)]
    terms_z = [(-tp * np.sin(tp * X) * np.sin(tp * Z), 1 + 1), (-tp * np.cos(tp * Y) * np.sin(2 * tp * Z), 1 + 4)]
    u = np.stack([sum(-t / (tp * tp * k2) for t, k2 in T) for T in (terms_x, terms_y, terms_z)])
    bc = (((PER, PER),) * 3,) * 3
    out = oracle.biot_savart(f, bc, (h, h, h), center=CELL, kernel="spectral")
    assert np.abs(out - u).max() < 1e-13


def test_biot_savart_symmetric_unbounded_matches_scalar_solves():
    """Vorticity tube f = (0, 0, w(x, y)) with x, y unbounded and z even: u_x solves
    lap = dw/dy, u_y solves lap = -dw/dx, with the derivatives taken analytically."""
    N = 16
    h = 1.0 / N
    x = np.arange(N + 1) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    s = 0.08
    w = np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / (2 * s * s))
    f = np.stack([0 * w, 0 * w, w])
    bc = (((UNB, UNB), (UNB, UNB), (ODD, ODD)), ((UNB, UNB), (UNB, UNB), (ODD, ODD)), ((UNB, UNB), (UNB, UNB), (EVEN, EVEN)))
    out = oracle.biot_savart(f, bc, (h, h, h), center=NODE, kernel="hej2")
    bcu = oracle.curl_bc(bc)
    assert bcu[0][2] == (EVEN, EVEN) and bcu[2][2] == (ODD, ODD)
    dwdy = -(Y - 0.5) / (s * s) * w
    dwdx = -(X - 0.5) / (s * s) * w
    ux = solve(dwdy, Problem(bc=bcu[0], h=(h, h, h), center=NODE, kernel="hej2"))
    uy = solve(-dwdx, Problem(bc=bcu[1], h=(h, h, h), center=NODE, kernel="hej2"))
    scale = np.abs(ux).max()
    # the spectral derivative of the (well-resolved, 10 sigma wide) Gaussian is exact to ~1e-6
    assert np.abs(out[0] - ux).max() < 2e-3 * scale
    assert np.abs(out[1] - uy).max() < 2e-3 * scale
    assert np.abs(out[2]).max() < 1e-14


# ---------------------------------------------------------------------------
# Finite-difference derivative symbols of the Biot-Savart curl (Section
# "Biot-Savart solver": orders 2, 4 and 6) against real-space central
# differences with the textbook stencil weights, and against their order.
# ---------------------------------------------------------------------------
_STENCILS = {"fd2": (1.0 / 2.0,), "fd4": (2.0 / 3.0, -1.0 / 12.0), "fd6": (3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0)}


def _curl_stencil(f, h, weights):
    """Curl of a periodic [c, z, y, x] field, d/dx_d a = sum_m w_m (a_{j+m} - a_{j-m}) / h_d."""
    def d(a, direction):
        ax = 2 - direction
        out = np.zeros_like(a)
        for m, w in enumerate(weights, start=1):
            out += w * (np.roll(a, -m, axis=ax) - np.roll(a, m, axis=ax)) / h[direction]
        return out
    fx, fy, fz = f
    return np.stack([d(fz, 1) - d(fy, 2), d(fx, 2) - d(fz, 0), d(fy, 0) - d(fx, 1)])


@pytest.mark.parametrize("diff", ["fd2", "fd4", "fd6"])
def test_finite_difference_curl_is_the_central_stencil(diff):
    """Periodic grid: u of the FD Biot-Savart solve = the Poisson solves of the stencil curl."""
    rng = np.random.default_rng(61)
    f = rng.standard_normal((3, 8, 12, 16))
    h = (1.0 / 16, 1.0 / 12, 1.0 / 8)
    bc = ((PER, PER),) * 3
    u = oracle.biot_savart(f, (bc, bc, bc), h, center=CELL, kernel="spectral", diff=diff)
    c = _curl_stencil(f, h, _STENCILS[diff])
    want = np.stack([solve(c[i], Problem(bc=bc, h=h, center=CELL, kernel="spectral")) for i in range(3)])
    assert np.abs(u - want).max() < 1e-13 * np.abs(want).max()


def test_finite_difference_orders():
    """A smooth periodic field: the FD velocity approaches the spectral one as h^2, h^4, h^6."""
    def field(n):
        x = (np.arange(n) + 0.5) / n
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        s = 2 * math.pi
        return np.stack([np.sin(s * Y) * np.cos(s * Z), np.sin(s * Z) * np.cos(2 * s * X), np.cos(s * X) * np.sin(s * Y)])
    bc = ((PER, PER),) * 3
    errs = {k: [] for k in _STENCILS}
    for n in (32, 64):
        f = field(n)
        h = (1.0 / n,) * 3
        ref = oracle.biot_savart(f, (bc, bc, bc), h, center=CELL, kernel="spectral", diff="spectral")
        for k in _STENCILS:
            u = oracle.biot_savart(f, (bc, bc, bc), h, center=CELL, kernel="spectral", diff=k)
            errs[k].append(np.abs(u - ref).max())
    for k, p in (("fd2", 2), ("fd4", 4), ("fd6", 6)):
        rate = math.log2(errs[k][0] / errs[k][1])
        assert abs(rate - p) < 0.1, (k, rate)
