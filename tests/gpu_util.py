"""Helpers of the GPU tests: run the CUDA path through the C ABI binding."""
import numpy as np

from paper_2211_07777_gb300 import flups as F


def cuda_solve(f, bc, center, prec, kernel, L=(1.0, 1.0, 1.0), eps_over_h=2.0, op=F.POISSON, diff=0, in_place=False,
               h=None):
    """Solve on the GPU; f is float64 [z, y, x] (or [c, z, y, x]); returns float64 numpy."""
    import torch
    n = (f.shape[-1], f.shape[-2], f.shape[-3])
    ncomp = 3 if f.ndim == 4 else 1
    dt = torch.float32 if prec == F.F32 else torch.float64
    s = F.Solver(n, bc, L=L, center=center, prec=prec, green=kernel, eps_over_h=eps_over_h, op=op, diff=diff,
                 ncomp=ncomp, h=h)
    try:
        rhs = torch.from_numpy(np.ascontiguousarray(f)).to(device="cuda", dtype=dt)
        phi = rhs if in_place else torch.empty_like(rhs)
        s.solve(phi, rhs)
        torch.cuda.synchronize()
        code = s.check()
        assert code == 0, f"a bounded device wait gave up (code {code})"
        return phi.double().cpu().numpy(), s.info
    finally:
        s.close()


def rel_linf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
