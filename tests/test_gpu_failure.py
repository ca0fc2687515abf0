"""Device-side failure reporting, exercised without faulting the GPU.

The column passes and the fused pass wait on mbarriers for their TMA copies
(the input tile: code 2; the Green slice: code 1).  The test hook
flups_debug_wait_limit makes those waits give up at once, as a copy that never
arrived would; the copies themselves do arrive (the kernel drains them before
it exits), so nothing is left in flight.  The code must reach the host through
flups_solver_check (own workspace) and through the workspace's status word
(caller workspace, as the serving runtime uses), and the next normal solve must
be correct again.
"""
import numpy as np
import pytest

import oracle
from paper_2211_07777_gb300 import flups as F
from paper_2211_07777_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N = 128   # FP32 unbounded 128^3: compile-time column passes with TMA input tiles and a TMA Green slice


def _problem():
    f = W.gaussian_blob((N, N, N), 0.1, W.blob_center(2))
    bc = ((F.UNB, F.UNB),) * 3
    return f, bc


def _uses_both_waits(s):
    feats = s.features()
    return any(x["tma_green"] for x in feats) and any(x["tma_input"] for x in feats)


@pytest.fixture(scope="module")
def reference():
    f, _ = _problem()
    prob = oracle.Problem(bc=((oracle.UNB, oracle.UNB),) * 3, h=(1.0 / N,) * 3, center=oracle.CELL, kernel="hej2")
    return oracle.solve(f, prob)


@pytest.mark.parametrize("mask,code", [(1, 1), (2, 2)], ids=["green-slice", "input-tile"])
def test_wait_that_gives_up_is_reported_and_next_solve_is_valid(mask, code, reference):
    import torch
    f, bc = _problem()
    with F.Solver((N, N, N), bc, prec=F.F32, green="hej2") as s:
        assert _uses_both_waits(s)
        rhs = torch.from_numpy(f).to("cuda", torch.float32)
        phi = torch.zeros_like(rhs)
        s.debug_wait_limit(mask)
        s.solve(phi, rhs)
        torch.cuda.synchronize()
        assert s.check() == code
        assert s.check() == 0                      # the check resets the code
        s.debug_wait_limit(0)
        s.solve(phi, rhs)
        torch.cuda.synchronize()
        assert s.check() == 0
        got = phi.double().cpu().numpy()
        assert np.abs(got - reference).max() <= 1e-5 * np.abs(reference).max()


def test_workspace_status_word_reports_its_own_solve(reference):
    import torch
    f, bc = _problem()
    t = F.flups_init_topo((N, N, N), F.CELL, 1, F.F32)
    s = F.flups_init_solver(t, bc, [1.0 / N] * 3, [1.0] * 3, F.HEJ2)
    try:
        F.flups_setup_shared(s)
        nbytes = F.flups_workspace_size(s)
        off = F.flups_workspace_status(s)
        assert off % 4 == 0 and off + 4 <= nbytes
        ws_a = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        ws_b = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        ws_a[off:off + 4].fill_(0x7f)                  # garbage left by an earlier user: the solve zeroes it
        rhs = torch.from_numpy(f).to("cuda", torch.float32)
        phi_a, phi_b = torch.zeros_like(rhs), torch.zeros_like(rhs)

        def status(ws):
            return int(ws[off:off + 4].view(torch.int32).item())

        F.flups_debug_wait_limit(s, 1)
        F.flups_solve_ws(s, phi_b, rhs, ws_b)
        F.flups_debug_wait_limit(s, 0)
        F.flups_solve_ws(s, phi_a, rhs, ws_a)
        torch.cuda.synchronize()
        assert status(ws_b) == 1
        assert status(ws_a) == 0
        got = phi_a.double().cpu().numpy()
        assert np.abs(got - reference).max() <= 1e-5 * np.abs(reference).max()
    finally:
        F.flups_cleanup(s)
        F.flups_topo_free(t)
