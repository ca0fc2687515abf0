"""Parity at the benchmark configurations' full sizes, in the launch
configuration bench.py times (same solver, same tile shapes).

Full oracle comparisons where the oracle fits (periodic 32^3, unbounded 128^3,
mixed 257 x 256 x 257); at 512^3 and 1024^3, outputs the oracle computes one
by one (direct sums of the HEJ2 kernel) and closed forms that hold at any
size (sine products: phi = -f/|k|^2 per mode; Gaussian blob: the potential
of the eps-smoothed Gaussian).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import CELL, NODE, EVEN as E, ODD as O, PER, UNB as U
from paper_2211_07777_gb300 import flups as F
from paper_2211_07777_gb300 import workloads as W
from tests import analytic
from tests.gpu_util import cuda_solve, rel_linf

pytestmark = pytest.mark.gpu


def test_periodic_32_fp64_against_oracle_and_closed_form():
    n = 32
    modes = W.sine_modes(1)
    f = W.periodic_sines((n, n, n), modes)
    h = 1.0 / n
    ref = oracle.solve(f, oracle.Problem(bc=((PER, PER),) * 3, h=(h, h, h), center=CELL, kernel="spectral"))
    out, _ = cuda_solve(f, ((PER, PER),) * 3, CELL, F.F64, "spectral")
    assert rel_linf(out, ref) < 1e-12
    x = W.coords(n, 1.0, CELL)
    exact = np.zeros_like(f)
    for a, b, c, A in modes:
        exact += -A / ((2 * math.pi) ** 2 * (a * a + b * b + c * c)) * np.sin(2 * math.pi * c * x)[:, None, None] \
            * np.sin(2 * math.pi * b * x)[None, :, None] * np.sin(2 * math.pi * a * x)[None, None, :]
    assert rel_linf(out, exact) < 1e-12


@pytest.mark.parametrize("prec", [F.F64, F.F32], ids=["f64", "f32"])
def test_unbounded_128_against_oracle_and_direct_sums(prec):
    n = 128
    h = 1.0 / n
    c = W.blob_center(2)
    f = W.gaussian_blob((n, n, n), 0.1, c)
    ref = oracle.solve(f, oracle.Problem(bc=((U, U),) * 3, h=(h, h, h), center=CELL, kernel="hej2"))
    out, _ = cuda_solve(f, ((U, U),) * 3, CELL, prec, "hej2")
    assert rel_linf(out, ref) < (1e-12 if prec == F.F64 else 1e-5)
    # sampled outputs, one direct sum each: phi_i = h^3 sum_j G(|x_i - x_j|) f_j
    x = W.coords(n, 1.0, CELL)
    rng = np.random.default_rng(0)
    scale = np.abs(ref).max()
    for _ in range(6):
        i = rng.integers(0, n, size=3)
        dz = (x - x[i[0]])[:, None, None]
        dy = (x - x[i[1]])[None, :, None]
        dx = (x - x[i[2]])[None, None, :]
        r = np.sqrt(dx * dx + dy * dy + dz * dz)
        val = h ** 3 * np.sum(oracle.green.hej2_3d(r, 2 * h) * f)
        assert abs(out[i[0], i[1], i[2]] - val) < (1e-12 if prec == F.F64 else 1e-5) * scale
    # closed form: the eps-smoothed Gaussian potential, up to the blob's truncation by the box
    xs = x[None, None, :] - c[0], x[None, :, None] - c[1], x[:, None, None] - c[2]
    rr = np.sqrt(xs[0] ** 2 + xs[1] ** 2 + xs[2] ** 2)
    pot = analytic.gaussian_potential(rr, math.sqrt(0.01 + (2 * h) ** 2))
    assert rel_linf(out, pot) < 2e-6


@pytest.mark.slow
@pytest.mark.parametrize("prec", [F.F64, F.F32], ids=["f64", "f32"])
def test_mixed_257x256x257_against_oracle(prec):
    """Node-centred, x even-even (DCT-I), y periodic stored without the duplicate node, z unbounded."""
    f = W.mixed_blob_modes()
    h = 1.0 / 256
    full = np.concatenate([f, f[:, :1, :]], axis=1)
    ref = oracle.solve(full, oracle.Problem(bc=((E, E), (PER, PER), (U, U)), h=(h, h, h), center=NODE,
                                            kernel="hej2"))[:, :256, :]
    out, _ = cuda_solve(f, ((E, E), (PER, PER), (U, U)), NODE, prec, "hej2", h=(h, h, h))
    assert rel_linf(out, ref) < (1e-12 if prec == F.F64 else 1e-5)


@pytest.mark.parametrize("prec", [F.F64, F.F32], ids=["f64", "f32"])
def test_mixed_odd_odd_variant_against_oracle(prec):
    """x odd-odd (DST-I) variant of the mixed case at 65 x 64 x 65."""
    f = W.mixed_blob_modes(n=(65, 64, 65), h=1.0 / 64)
    h = 1.0 / 64
    full = np.concatenate([f, f[:, :1, :]], axis=1)
    ref = oracle.solve(full, oracle.Problem(bc=((O, O), (PER, PER), (U, U)), h=(h, h, h), center=NODE,
                                            kernel="hej2"))[:, :64, :]
    out, _ = cuda_solve(f, ((O, O), (PER, PER), (U, U)), NODE, prec, "hej2", h=(h, h, h))
    assert rel_linf(out, ref) < (1e-12 if prec == F.F64 else 1e-5)


@pytest.mark.slow
def test_unbounded_512_fp32():
    """FP32 at 512^3 against the FP64 path, direct sums at sampled points, and the closed form."""
    import torch
    n = 512
    h = 1.0 / n
    c = W.blob_center(2)
    f = W.gaussian_blob((n, n, n), 0.1, c)
    out32, _ = cuda_solve(f, ((U, U),) * 3, CELL, F.F32, "hej2")
    out64, _ = cuda_solve(f, ((U, U),) * 3, CELL, F.F64, "hej2")
    scale = np.abs(out64).max()
    assert np.abs(out32 - out64).max() < 1e-5 * scale
    x = W.coords(n, 1.0, CELL)
    rng = np.random.default_rng(1)
    for _ in range(2):
        i = rng.integers(0, n, size=3)
        dz = (x - x[i[0]])[:, None, None]
        dy = (x - x[i[1]])[None, :, None]
        dx = (x - x[i[2]])[None, None, :]
        r = np.sqrt(dx * dx + dy * dy + dz * dz)
        val = h ** 3 * np.sum(oracle.green.hej2_3d(r, 2 * h) * f)
        assert abs(out64[i[0], i[1], i[2]] - val) < 1e-12 * scale
        assert abs(out32[i[0], i[1], i[2]] - val) < 1e-5 * scale
    zc = [0, 100, 256, 511]
    xs = x[None, None, :] - c[0], x[None, :, None] - c[1], x[zc][:, None, None] - c[2]
    rr = np.sqrt(xs[0] ** 2 + xs[1] ** 2 + xs[2] ** 2)
    pot = analytic.gaussian_potential(rr, math.sqrt(0.01 + (2 * h) ** 2))
    assert np.abs(out32[zc] - pot).max() < 3e-6 * scale


@pytest.mark.slow
def test_periodic_1024_fp64_closed_form_on_sampled_planes():
    import torch
    n = 1024
    modes = W.sine_modes(5)
    rhs = W.periodic_sines_torch((n, n, n), modes, "cuda", torch.float64)
    s = F.Solver((n, n, n), ((PER, PER),) * 3, prec=F.F64, green="spectral")
    try:
        phi = torch.empty_like(rhs)
        s.solve(phi, rhs)
        torch.cuda.synchronize()
        zidx = [0, 1, 333, 1023]
        out = phi[zidx].cpu().numpy()
    finally:
        s.close()
    del rhs, phi
    x = W.coords(n, 1.0, CELL)
    exact = np.zeros((len(zidx), n, n))
    for a, b, c, A in modes:
        exact += -A / ((2 * math.pi) ** 2 * (a * a + b * b + c * c)) * np.sin(2 * math.pi * c * x[zidx])[:, None, None] \
            * np.sin(2 * math.pi * b * x)[None, :, None] * np.sin(2 * math.pi * a * x)[None, None, :]
    amp = sum(abs(A) / ((2 * math.pi) ** 2 * (a * a + b * b + c * c)) for a, b, c, A in modes)
    assert np.abs(out - exact).max() < 1e-12 * amp
