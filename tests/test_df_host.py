"""The conversions between FP64 and double-float (hi + lo pairs of FP32 words) that the
double-float passes apply to the caller's FP64 arrays (csrc/dfloat.cuh), compiled for the host and
checked against exact rational arithmetic: hi + lo represents d to 2^-47 relative with |lo| <=
ulp(hi)/2, and the way back is the FP64 value nearest to hi + lo."""
import math
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2211_07777_gb300", "csrc")


@pytest.fixture(scope="module")
def df_exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("df") / "df_check")
    src = os.path.join(ROOT, "tests", "host", "df_check.cu")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, src, "-o", out], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return out


def _f32(b):
    return struct.unpack("<f", struct.pack("<I", b))[0]


def _f64(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def _bits(d):
    return struct.unpack("<Q", struct.pack("<d", d))[0]


def test_conversions_match_exact_arithmetic(df_exe):
    rng = np.random.default_rng(5)
    vals = list(rng.standard_normal(2000) * 10.0 ** rng.uniform(-20, 20, 2000))
    vals += [1.0, -1.0, 0.5, 3.0, 1.0 + 2.0 ** -52, 1.0 - 2.0 ** -53, 2.0 ** 127 * 1.5, 2.0 ** -74, -2.0 ** -74 * 1.25,
             math.pi, -math.e, 0.1, 1e-30, 0.0, -0.0, 2.0 ** -80, 1e-300, 5e-324]
    vals += [_f64(0x3FF0000000000000 | int(m)) for m in rng.integers(0, 2 ** 52, 200)]
    inp = "\n".join(f"{_bits(v):016x}" for v in vals) + "\n"
    r = subprocess.run([df_exe], input=inp, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.split("\n")
    for v, ln in zip(vals, lines):
        hb, lb, db = ln.split()
        hi, lo, back = _f32(int(hb, 16)), _f32(int(lb, 16)), _f64(int(db, 16))
        exact = Fraction(hi) + Fraction(lo)
        if v == 0.0:
            assert hi == 0.0 and lo == 0.0 and back == 0.0
            continue
        # hi + lo represents v to 2^-47 relative (float-range values; tinier ones keep at least hi)
        err = abs(exact - Fraction(v)) / abs(Fraction(v))
        bound = 2.0 ** -47 if abs(v) >= 2.0 ** -74 else 2.0 ** -20
        if abs(v) >= 2.0 ** -126:
            assert err <= bound, (v, hi, lo, float(err))
        # normalised pair: |lo| <= ulp(hi) / 2
        if hi != 0.0 and math.isfinite(hi):
            ulp = 2.0 ** (math.frexp(hi)[1] - 24)
            assert abs(lo) <= ulp / 2, (v, hi, lo)
        # the way back: the double nearest to hi + lo
        assert back == float(exact), (v, hi, lo, back)
