"""Edge cases of the CUDA path against the oracle: the longest transform (4096 points, doubled
and semi-unbounded), the smallest grids (N = 4), and degenerate right-hand sides."""
import numpy as np
import pytest

import oracle
from oracle import CELL, NODE, EVEN as E, ODD as O, PER, UNB as U
from paper_2211_07777_gb300 import flups as F
from tests.gpu_util import cuda_solve, rel_linf

pytestmark = pytest.mark.gpu

TOL = {F.F64: 1e-12, F.F32: 1e-5, F.F64E: 1e-12}
PRECS = [F.F64, F.F32, F.F64E]
IDS = ["f64", "f32", "f64e"]


def _case(shape, bc, center, kernel, seed):
    rng = np.random.default_rng(seed)
    f = rng.standard_normal(shape)
    n = (shape[2], shape[1], shape[0])
    h = tuple(1.0 / (n[d] if center == CELL else n[d] - 1) for d in range(3))
    ref = oracle.solve(f, oracle.Problem(bc=bc, h=h, center=center, kernel=kernel))
    return f, ref


@pytest.mark.parametrize("prec", PRECS, ids=IDS)
@pytest.mark.parametrize("bc,shape", [
    (((U, U), (PER, PER), (E, E)), (8, 8, 2048)),    # x doubled: 4096 points
    (((U, E), (O, O), (PER, PER)), (8, 8, 1024)),    # x semi-unbounded: 4 x 1024 points
], ids=["unb-4096", "semi-4096"])
def test_longest_transform(bc, shape, prec):
    f, ref = _case(shape, bc, CELL, "hej2", 61)
    out, _ = cuda_solve(f, bc, CELL, prec, "hej2")
    assert rel_linf(out, ref) < TOL[prec], rel_linf(out, ref)


@pytest.mark.parametrize("prec", PRECS, ids=IDS)
@pytest.mark.parametrize("center", [CELL, NODE], ids=["cell", "node"])
@pytest.mark.parametrize("bc", [((PER, PER), (U, U), (E, O)), ((O, E), (U, E), (O, U)), ((U, U),) * 3],
                         ids=["per-unb-eo", "oe-ue-ou", "unb"])
def test_smallest_grids(bc, center, prec):
    shape = (4, 4, 4) if center == CELL else (5, 5, 5)
    f, ref = _case(shape, bc, center, "hej2", 62)
    out, _ = cuda_solve(f, bc, center, prec, "hej2")
    assert rel_linf(out, ref) < TOL[prec], rel_linf(out, ref)


@pytest.mark.parametrize("prec", PRECS, ids=IDS)
def test_zero_right_hand_side_gives_zero(prec):
    f = np.zeros((8, 12, 16))
    out, _ = cuda_solve(f, ((U, U), (PER, PER), (E, O)), CELL, prec, "hej2")
    assert np.all(out == 0.0)


@pytest.mark.parametrize("prec", PRECS, ids=IDS)
def test_constant_right_hand_side_periodic_is_the_zero_mode(prec):
    """Fully periodic: the spectral kernel's zero mode is 0, so a constant right-hand side
    (pure zero mode) gives phi = 0 to rounding."""
    f = np.full((16, 16, 32), 3.0)
    out, _ = cuda_solve(f, ((PER, PER),) * 3, CELL, prec, "spectral")
    assert np.abs(out).max() < (1e-5 if prec == F.F32 else 1e-12)


_LONG = {}


@pytest.mark.parametrize("prec", PRECS, ids=IDS)
def test_longest_column_transform(prec):
    """z unbounded with 1024 cells: the fused column pass runs the compile-time tile at P = 2048
    (4 lanes FP32, 2 lanes FP64 and double-float), fed by TMA where that applies."""
    shape = (1024, 64, 64)
    bc = ((PER, PER), (PER, PER), (U, U))
    if not _LONG:
        _LONG["case"] = _case(shape, bc, CELL, "hej2", 63)
    f, ref = _LONG["case"]
    out, _ = cuda_solve(f, bc, CELL, prec, "hej2")
    assert rel_linf(out, ref) < TOL[prec], rel_linf(out, ref)
