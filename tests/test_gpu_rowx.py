"""The x passes on the register-chained stages (periodic and doubled unbounded x, FP32 and
double-float, 1024-point transforms) against the FP64 oracle, and the generic row kernels the same solve uses when its
arrays are pinned host memory.  The grids have few y-z rows but enough for the compile-time
engine: 1024 (periodic) or 512 doubled (unbounded) points along x."""
import numpy as np
import pytest

import oracle
from paper_2211_07777_gb300 import flups as F
from paper_2211_07777_gb300 import workloads as W
from tests.gpu_util import rel_linf

pytestmark = pytest.mark.gpu

P, U = F.PER, F.UNB

CASES = [
    ((1024, 64, 48), ((P, P), (P, P), (P, P)), "spectral"),
    ((512, 64, 48), ((U, U), (U, U), (U, U)), "hej2"),
    ((1024, 48, 64), ((P, P), (U, U), (P, P)), "hej2"),
]


def _rhs(n, seed):
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((n[2], n[1], n[0]))
    return f - f.mean()


_REFS = {}


def _reference(n, bc, kernel):
    key = (n, bc, kernel)
    if key not in _REFS:
        f = _rhs(n, sum(n))
        hh = (1.0 / n[0],) * 3
        _REFS[key] = (f, oracle.solve(f, oracle.Problem(bc=bc, h=hh, center=oracle.CELL, kernel=kernel)))
    return _REFS[key]


@pytest.mark.parametrize("prec", [F.F32, F.F64E], ids=["f32", "f64e"])
@pytest.mark.parametrize("n,bc,kernel", CASES, ids=["periodic", "unbounded", "periodic-x-unbounded-y"])
def test_row_stages_match_the_oracle(n, bc, kernel, prec):
    import torch
    f, ref = _reference(n, bc, kernel)
    L = tuple(v / n[0] for v in n)
    tol, tol_same = (1e-5, 2e-6) if prec == F.F32 else (1e-12, 1e-13)
    dt = torch.float32 if prec == F.F32 else torch.float64
    with F.Solver(n, bc, L=L, center=F.CELL, prec=prec, green=kernel) as s:
        feats = s.features()
        assert feats[0]["row_stages"] and feats[-1]["row_stages"], feats
        rhs = torch.from_numpy(f).to("cuda", dt)
        phi = torch.empty_like(rhs)
        s.solve(phi, rhs)
        torch.cuda.synchronize()
        assert s.check() == 0
        dev = phi.double().cpu().numpy()
        assert rel_linf(dev, ref) < tol
        # pinned host arrays: the kernels read and write them across the host link with the
        # generic row kernels; the same result to rounding
        h_in = torch.from_numpy(f.astype(np.float32 if prec == F.F32 else np.float64)).pin_memory()
        h_out = torch.zeros_like(h_in).pin_memory()
        s.solve_host(h_out, h_in)
        assert s.check() == 0
        host = h_out.double().numpy()
        assert rel_linf(host, ref) < tol
        assert rel_linf(host, dev) < tol_same
