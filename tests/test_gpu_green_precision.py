"""Precision of the stored Green's function spectrum.

The setup samples the kernel in FP64 on the device and transforms it along
every unbounded-like direction with the DCT-I of the kernel symmetrised on the
extended domain (Section 2.3: the Green's function is evaluated on the doubled
or padded domain and Fourier transformed there).  Those transforms run in
double-float arithmetic on the FP32 units.  This test reads the device's own
FP64 samples and the stored spectrum back (flups_debug_green) and redoes the
transform in FP64 with NumPy from the definition of the DCT-I (Section 2.2.1):
X_k = g_0 + (-1)^k g_M + 2 sum_{j=1}^{M-1} g_j cos(pi j k / M), computed as the
DFT of the even extension.  The stored FP64 spectrum must agree to 1e-13
relative; an FP32 one to its rounding (1e-7).
"""
import numpy as np
import pytest

from paper_2211_07777_gb300 import flups as F

pytestmark = pytest.mark.gpu

E, O, P, U = F.EVEN, F.ODD, F.PER, F.UNB


def _period(n_data, bc, center):
    """Extended period P of a direction and whether it is unbounded-like (sampled in real space)."""
    l, r = bc
    N = n_data if center == F.CELL else n_data - 1
    if l == P:
        return N, False
    if l == U and r == U:
        return 2 * N, True
    if U in (l, r):
        return 4 * N, True
    return (2 * N if l == r else 4 * N), False


def _dct1(a, axis):
    """DCT-I along `axis` (M + 1 samples): the DFT of the even extension, real part, first M + 1."""
    a = np.moveaxis(a, axis, -1)
    ext = np.concatenate([a, a[..., -2:0:-1]], axis=-1)
    out = np.fft.fft(ext, axis=-1).real[..., :a.shape[-1]]
    return np.moveaxis(out, -1, axis)


CASES = [
    ((32, 32, 32), ((U, U), (U, U), (U, U)), F.CELL, F.F64, "hej2", 1e-13),
    ((48, 32, 24), ((U, U), (P, P), (E, U)), F.CELL, F.F64, "hej4", 1e-13),
    ((33, 17, 33), ((U, U), (O, O), (U, U)), F.NODE, F.F64, "hej2", 1e-13),
    ((64, 64, 64), ((U, U), (U, U), (U, U)), F.CELL, F.F32, "hej6", 1e-7),
    ((32, 32, 32), ((U, U), (U, U), (U, U)), F.CELL, F.F64E, "lgf2", 1e-13),
]


@pytest.mark.parametrize("n,bc,center,prec,kernel,tol", CASES,
                         ids=["unb32-f64-hej2", "mixed-semi-f64-hej4", "node-f64-hej2", "unb64-f32-hej6",
                              "unb32-df-lgf2"])
def test_stored_spectrum_is_the_fp64_transform_of_the_samples(n, bc, center, prec, kernel, tol):
    s = F.Solver(n, bc, center=center, prec=prec, green=kernel)
    try:
        periods, unb, h = [], [], []
        for d in range(3):
            Pd, ud = _period(n[d], bc[d], center)
            periods.append(Pd)
            unb.append(ud)
            h.append(1.0 / (n[d] if center == F.CELL else n[d] - 1))
        # Green index extents: an unbounded-like direction holds P/2 + 1 samples r = g h; a spectral
        # one its folded modes (periodic N/2 + 1, half-wave N + 1, quarter-wave N)
        ext = [periods[d] // 2 + 1 if unb[d] else _modes(n[d], bc[d], center) for d in range(3)]
        samples, spectrum = F.flups_debug_green(s._s, int(np.prod(ext)))
        shape = (ext[2], ext[1], ext[0])
        g = samples.reshape(shape)
        want = g
        for d in range(3):
            if unb[d]:
                want = _dct1(want, 2 - d)
        want = want * np.prod([h[d] for d in range(3) if unb[d]]) / np.prod(periods)
        got = spectrum.reshape(shape)
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err <= tol, err
    finally:
        s.close()


def _modes(n_data, bc, center):
    N = n_data if center == F.CELL else n_data - 1
    l, r = bc
    if l == P:
        return N // 2 + 1
    return N + 1 if l == r else N
