"""Convergence orders of the CUDA Biot-Savart solve on the paper's vortex tube.

Section "Application: the Biot-Savart solver": a compact vortex tube along z
(x and y unbounded; z symmetric, the x and y vorticity components odd and the z
component even), compared with its closed-form velocity; the measured order is
the minimum of the differentiation order and the kernel order.  The radius is
not given (its printed E_inf stay unpinned); R = 0.4 L here.  Node-centred,
N = 128 ... 1024 in x and y (the field does not depend on z: 4 cells there).
The orders at the finest pair (measured on a GB300): HEJ2 2.00 with every
derivative; FD2 2.00 with HEJ4; HEJ4 with FD4 3.90; HEJ6 with FD6 5.70; HEJ8
with FD4 4.22 -- each within a margin of min(derivative order, kernel order).
"""
import math

import numpy as np
import pytest

from paper_2211_07777_gb300 import flups as F
from tests.analytic import vortex_tube

pytestmark = pytest.mark.gpu

E, O, U = F.EVEN, F.ODD, F.UNB
BC_F = (((U, U), (U, U), (O, O)), ((U, U), (U, U), (O, O)), ((U, U), (U, U), (E, E)))
R = 0.4
NS = (128, 256, 512, 1024)


def _errors(kernel, diff):
    import torch
    errs = []
    for N in NS:
        f, u = vortex_tube(N, 4, R)
        s = F.Solver((N + 1, N + 1, 5), BC_F, L=(1.0, 1.0, 4.0 / N), center=F.NODE, prec=F.F64, green=kernel,
                     op=F.BIOT_SAVART, diff=diff, ncomp=3)
        try:
            rhs = torch.from_numpy(f).to("cuda", torch.float64)
            phi = torch.empty_like(rhs)
            s.solve(phi, rhs)
            torch.cuda.synchronize()
            assert s.check() == 0
            errs.append(float(np.abs(phi.cpu().numpy() - u).max()))
        finally:
            s.close()
    return errs


# (kernel, derivative, expected order min(d, k), accepted range of the finest-pair order)
CASES = [
    ("hej2", F.DIFF_SPECTRAL, 2, (1.9, 2.1)),
    ("hej2", F.DIFF_FD6, 2, (1.9, 2.1)),
    ("hej4", F.DIFF_FD2, 2, (1.9, 2.1)),
    ("hej4", F.DIFF_FD4, 4, (3.7, 4.3)),
    ("hej6", F.DIFF_FD6, 6, (5.4, 6.4)),
    ("hej8", F.DIFF_FD4, 4, (3.6, 4.7)),
]


@pytest.mark.parametrize("kernel,diff,order,bounds", CASES,
                         ids=[f"{k}-d{d}" for k, d, _, _ in CASES])
def test_order_is_min_of_derivative_and_kernel(kernel, diff, order, bounds):
    errs = _errors(kernel, diff)
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert bounds[0] <= orders[-1] <= bounds[1], (errs, orders)
    assert errs[-1] < errs[0]
