"""Biot-Savart (lap u = curl f) on the GPU against the oracle, element by element."""
import numpy as np
import pytest

import oracle
from oracle import CELL, NODE, EVEN as E, ODD as O, PER, UNB as U
from paper_2211_07777_gb300 import flups as F
from tests.gpu_util import cuda_solve, rel_linf

pytestmark = pytest.mark.gpu

PAIRS = {"PER": (PER, PER), "UNB": (U, U), "EE": (E, E), "OO": (O, O), "EO": (E, O), "OE": (O, E),
         "EU": (E, U), "OU": (O, U), "UE": (U, E), "UO": (U, O)}


def swap(b):
    return {E: O, O: E}.get(b, b)


def wall_rule(dirs):
    """Face conditions of the three components: component d takes the swapped parity along d."""
    out = []
    for c in range(3):
        comp = []
        for d in range(3):
            l, r = PAIRS[dirs[d]]
            comp.append((swap(l), swap(r)) if c == d else (l, r))
        out.append(tuple(comp))
    return tuple(out)


def _cases():
    rng = np.random.default_rng(2156)
    names = list(PAIRS)
    cases = [("UNB", "UNB", "OO"), ("PER", "PER", "PER"), ("UNB", "UNB", "UNB"), ("EE", "OE", "PER")]
    for _ in range(10):
        cases.append(tuple(rng.choice(names, size=3)))
    return cases


CASES = _cases()
_CACHE = {}


def _ref(dirs, center, diff):
    key = (dirs, center, diff)
    if key not in _CACHE:
        shape = (8, 12, 16) if center == CELL else (9, 13, 17)
        rng = np.random.default_rng(sum(map(ord, "".join(dirs))) + 1000 * center)
        f = rng.standard_normal((3,) + shape)
        n = (shape[2], shape[1], shape[0])
        h = tuple(1.0 / (n[d] if center == CELL else n[d] - 1) for d in range(3))
        kernel = "hej2" if any("U" in t for t in dirs) else "spectral"
        bcf = wall_rule(dirs)
        u = oracle.biot_savart(f, bcf, h, center=center, kernel=kernel, diff=diff)
        _CACHE[key] = (f, bcf, kernel, u)
    return _CACHE[key]


@pytest.mark.parametrize("prec", [F.F64, F.F32, F.F64E], ids=["f64", "f32", "f64e"])
@pytest.mark.parametrize("center", [CELL, NODE], ids=["cell", "node"])
@pytest.mark.parametrize("dirs", CASES, ids=["-".join(c) for c in CASES])
def test_biot_savart_matches_oracle(dirs, center, prec):
    f, bcf, kernel, ref = _ref(dirs, center, "spectral")
    out, _ = cuda_solve(f, bcf, center, prec, kernel, op=F.BIOT_SAVART)
    tol = 1e-5 if prec == F.F32 else 1e-12
    assert rel_linf(out, ref) < tol, rel_linf(out, ref)


@pytest.mark.parametrize("diff", ["fd2", "fd4", "fd6"])
@pytest.mark.parametrize("dirs", [("UNB", "UNB", "OO"), ("PER", "EE", "UNB"), ("OU", "PER", "EO")],
                         ids=["tube", "per-ee-unb", "ou-per-eo"])
def test_biot_savart_finite_difference_symbols(dirs, diff):
    f, bcf, kernel, ref = _ref(dirs, CELL, diff)
    code = {"fd2": F.DIFF_FD2, "fd4": F.DIFF_FD4, "fd6": F.DIFF_FD6}[diff]
    out, _ = cuda_solve(f, bcf, CELL, F.F64, kernel, op=F.BIOT_SAVART, diff=code)
    assert rel_linf(out, ref) < 1e-12


def test_biot_savart_rejects_inconsistent_vector_conditions():
    bcf = wall_rule(("UNB", "UNB", "OO"))
    bad = (bcf[0], bcf[1], ((U, U), (U, U), (O, O)))   # normal component not flipped
    with pytest.raises(F.FlupsError) as e:
        F.Solver((16, 16, 16), bad, op=F.BIOT_SAVART, green="hej2")
    assert e.value.status == -2
