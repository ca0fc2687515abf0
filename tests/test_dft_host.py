"""The FFT engine's register DFTs (radix 2, 3, 4, 8, 16, 32, and the half-zero DFT-4 and DFT-32
used on zero-padded inputs), compiled for the host and checked against the definition of the DFT
(numpy's FFT) in FP64 -- the butterflies every pass kernel is built from, checked without a GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2211_07777_gb300", "csrc")


@pytest.fixture(scope="module")
def dft_exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("dft") / "dft_check")
    src = os.path.join(ROOT, "tests", "host", "dft_check.cu")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-I", os.path.join(ROOT, "include"), src, "-o", out],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return out


def _run(exe, cases):
    lines = []
    for R, inv, zh, x in cases:
        lines.append(f"{R} {int(inv)} {int(zh)} {len(x)}")
        lines += [f"{float(v.real):.17g} {float(v.imag):.17g}" for v in x]
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    vals = np.array([[float(t) for t in ln.split()] for ln in r.stdout.split("\n") if ln.strip()])
    return vals[:, 0] + 1j * vals[:, 1]


@pytest.mark.parametrize("inv", [False, True], ids=["forward", "inverse"])
def test_register_dfts_match_the_definition(dft_exe, inv):
    rng = np.random.default_rng(7)
    cases, want = [], []
    for R in (2, 3, 4, 8, 16, 32):
        for _ in range(3):
            x = rng.standard_normal(R) + 1j * rng.standard_normal(R)
            cases.append((R, inv, False, x))
            want.append(np.fft.ifft(x) * R if inv else np.fft.fft(x))
    got = _run(dft_exe, cases)
    want = np.concatenate(want)
    assert np.abs(got - want).max() < 1e-14 * np.abs(want).max()


@pytest.mark.parametrize("inv", [False, True], ids=["forward", "inverse"])
def test_half_zero_dfts_match_the_definition(dft_exe, inv):
    """dft4_half(a, b) is the DFT-4 of (a, b, 0, 0); dft32 with ZH is the DFT-32 of 16 values then
    16 zeros (the first stage of a transform whose second half is zero padding)."""
    rng = np.random.default_rng(8)
    cases, want = [], []
    for R, nz in ((44, 2), (32, 16)):
        m = 4 if R == 44 else R
        for _ in range(3):
            x = np.zeros(m, complex)
            x[:nz] = rng.standard_normal(nz) + 1j * rng.standard_normal(nz)
            # the engine's input for the zero half is ignored: fill it with garbage
            xin = x.copy()
            xin[nz:] = 1e3 * (rng.standard_normal(m - nz) + 1j * rng.standard_normal(m - nz))
            cases.append((R, inv, True, xin))
            want.append(np.fft.ifft(x) * m if inv else np.fft.fft(x))
    got = _run(dft_exe, cases)
    want = np.concatenate(want)
    assert np.abs(got - want).max() < 1e-14 * np.abs(want).max()
