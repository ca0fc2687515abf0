"""The double-float (FP64-class, FP32-unit) path against the oracle at the FP64 tolerance."""
import json
import os
import zlib

import numpy as np
import pytest

import oracle
from oracle import CELL, NODE, EVEN as E, ODD as O, PER, UNB as U
from paper_2211_07777_gb300 import flups as F
from paper_2211_07777_gb300 import workloads as W
from tests import analytic
from tests.gpu_util import cuda_solve, rel_linf
from tests.test_gpu_parity import CASES, TYPES, _kernel

pytestmark = pytest.mark.gpu

_CACHE = {}


def _cells(t):
    """Cells per direction so that every transform length (N, 2N or 4N) is 32."""
    return 32 if t == "PER" else (16 if t in ("UNB", "EE", "OO") else 8)


def _ref(types, center):
    key = (types, center)
    if key not in _CACHE:
        N = [_cells(t) for t in types]
        shape = tuple(N[d] + (0 if center == CELL else 1) for d in (2, 1, 0))
        rng = np.random.default_rng(zlib.crc32("-".join(types).encode()) % 1000 + 7)
        f = rng.standard_normal(shape)
        n = (shape[2], shape[1], shape[0])
        h = tuple(1.0 / (n[d] if center == CELL else n[d] - 1) for d in range(3))
        prob = oracle.Problem(bc=tuple(TYPES[t] for t in types), h=h, center=center, kernel=_kernel(types))
        _CACHE[key] = (f, oracle.solve(f, prob))
    return _CACHE[key]


@pytest.mark.parametrize("center", [CELL, NODE], ids=["cell", "node"])
@pytest.mark.parametrize("types", CASES, ids=["-".join(c) for c in CASES])
def test_double_float_sweep_matches_oracle(types, center):
    f, ref = _ref(types, center)
    out, _ = cuda_solve(f, tuple(TYPES[t] for t in types), center, F.F64E, _kernel(types))
    assert rel_linf(out, ref) < 1e-12, rel_linf(out, ref)


with open(os.path.join(os.path.dirname(__file__), "golden", "paper_einf.json")) as fh:
    _G = json.load(fh)


@pytest.mark.parametrize("kernel", ["spectral", "lgf2", "hej2", "hej6", "hej10"])
def test_double_float_printed_symmetric_periodic(kernel):
    phi, f = analytic.case_symmetric_periodic(32)
    out, _ = cuda_solve(f, ((E, E), (O, E), (PER, PER)), NODE, F.F64E, kernel)
    err = np.abs(out - phi).max()
    want = _G["symmetric_periodic"][kernel]["33"]
    if want < 1e-13:
        assert err < 1e-13
    else:
        assert abs(err - want) < 1e-10 * want


def test_double_float_printed_unbounded():
    phi, f = analytic.case_unbounded(32)
    out, _ = cuda_solve(f, ((U, U),) * 3, NODE, F.F64E, "hej2")
    want = _G["unbounded"]["hej2"]["33"]
    assert abs(np.abs(out - phi).max() - want) < 1e-10 * want


def test_double_float_unbounded_128_against_oracle():
    n = 128
    h = 1.0 / n
    f = W.gaussian_blob((n, n, n), 0.1, W.blob_center(2))
    ref = oracle.solve(f, oracle.Problem(bc=((U, U),) * 3, h=(h, h, h), center=CELL, kernel="hej2"))
    out, _ = cuda_solve(f, ((U, U),) * 3, CELL, F.F64E, "hej2")
    assert rel_linf(out, ref) < 1e-12


def test_double_float_accepts_what_the_other_paths_accept():
    """Sizes 2^a 3^b and the Biot-Savart operator build; sizes with other prime factors are
    refused with FLUPS_ESIZE as on every path."""
    F.Solver((24, 16, 16), ((PER, PER),) * 3, prec=F.F64E).close()
    F.Solver((16, 16, 16), (((PER, PER),) * 3,) * 3, prec=F.F64E, op=F.BIOT_SAVART).close()
    with pytest.raises(F.FlupsError) as e:
        F.Solver((20, 16, 16), ((PER, PER),) * 3, prec=F.F64E)
    assert e.value.status == -3


@pytest.mark.parametrize("types", CASES[::3], ids=["-".join(c) for c in CASES[::3]])
def test_double_float_transform_lengths_2a3b(types):
    """Lengths 2^a 3^b (here 12 cells: 12, 24 or 48 per transform) run on the runtime-shaped
    double-float tiles; small grids take them too."""
    shape = (8, 12, 16)
    rng = np.random.default_rng(zlib.crc32("-".join(types).encode()) % 1000 + 9)
    f = rng.standard_normal(shape)
    n = (shape[2], shape[1], shape[0])
    h = tuple(1.0 / n[d] for d in range(3))
    bc = tuple(TYPES[t] for t in types)
    ref = oracle.solve(f, oracle.Problem(bc=bc, h=h, center=CELL, kernel=_kernel(types)))
    out, _ = cuda_solve(f, bc, CELL, F.F64E, _kernel(types))
    assert rel_linf(out, ref) < 1e-12, rel_linf(out, ref)


def test_double_float_large_2a3b_against_fp64():
    """96 x 192 x 64 cells (P up to 384): the double-float path against the native FP64 path."""
    rng = np.random.default_rng(21)
    f = rng.standard_normal((64, 192, 96))
    bc = ((U, U), (PER, PER), (E, O))
    a, _ = cuda_solve(f, bc, CELL, F.F64E, "hej2")
    b, _ = cuda_solve(f, bc, CELL, F.F64, "hej2")
    assert rel_linf(a, b) < 1e-12, rel_linf(a, b)
