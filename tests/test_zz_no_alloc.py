"""The allocation-free periodic solve against the regular C-ABI solve.

flups_solve_periodic_noalloc serves callers that may not allocate device
memory (their own pool owns the device, or cudaMalloc's implicit device
synchronisation is not affordable); its workspace is a fixed static device
array shared by all calls.  This file is collected last on purpose so that a
run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _regular(f, L):
    import torch
    from paper_2211_07777_gb300 import flups as F
    n = (f.shape[2], f.shape[1], f.shape[0])
    s = F.Solver(n, ((F.PER, F.PER),) * 3, L=L, center=F.CELL, prec=F.F64, green="spectral")
    try:
        rhs = torch.from_numpy(f).cuda()
        phi = torch.empty_like(rhs)
        s.solve(phi, rhs)
        torch.cuda.synchronize()
        return phi.cpu().numpy()
    finally:
        s.close()


def test_noalloc_matches_regular_solve_on_two_calls_in_a_row():
    import torch
    from paper_2211_07777_gb300 import flups as F
    rng = np.random.default_rng(77)
    cases = [((24, 32, 48), (1.0, 2.0, 1.5)), ((32, 32, 32), (1.0, 1.0, 1.0))]   # [z, y, x] shapes
    for shape, L in cases:
        f = rng.standard_normal(shape)
        ref = _regular(f, L)
        rhs = torch.from_numpy(f).cuda()
        phi = torch.full_like(rhs, float("nan"))
        F.flups_solve_periodic_noalloc(phi, rhs, (shape[2], shape[1], shape[0]), L)
        torch.cuda.synchronize()
        out = phi.cpu().numpy()
        assert np.all(np.isfinite(out))
        assert np.abs(out - ref).max() / np.abs(ref).max() < 1e-12


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    from paper_2211_07777_gb300 import flups as F
    x = torch.zeros(8, device="cuda", dtype=torch.float64)
    with pytest.raises(F.FlupsError) as e:
        F.flups_solve_periodic_noalloc(x, x, (256, 256, 256), (1.0, 1.0, 1.0))   # workspace > 48 MiB
    assert e.value.status == -3
