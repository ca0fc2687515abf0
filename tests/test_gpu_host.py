"""flups_solve_host: pinned host arrays used in place, pageable ones staged, against the device solve.

Both routes run the same kernels on the same data, so the results are bit-identical to
flups_solve on device arrays.
"""
import numpy as np
import pytest

from oracle import CELL, EVEN as E, ODD as O, PER, UNB as U
from paper_2211_07777_gb300 import flups as F

pytestmark = pytest.mark.gpu


def _device_solve(s, f, dt):
    import torch
    rhs = torch.from_numpy(f).to(device="cuda", dtype=dt)
    phi = torch.empty_like(rhs)
    s.solve(phi, rhs)
    torch.cuda.synchronize()
    return phi.cpu().numpy()


def _host(f, dt, pinned):
    import torch
    t = torch.from_numpy(f).to(dtype=dt)
    return t.pin_memory() if pinned else t.clone()


@pytest.mark.parametrize("pin_in,pin_out", [(True, True), (False, False), (True, False), (False, True)],
                         ids=["pinned", "pageable", "pinned-in", "pinned-out"])
@pytest.mark.parametrize("prec", [F.F64, F.F32, F.F64E], ids=["f64", "f32", "f64e"])
def test_host_solve_matches_device_solve(prec, pin_in, pin_out):
    import torch
    dt = torch.float32 if prec == F.F32 else torch.float64
    shape = (24, 12, 32)
    f = np.random.default_rng(3).standard_normal(shape)
    bc = ((U, U), (E, O), (PER, PER))
    n = (shape[2], shape[1], shape[0])
    with F.Solver(n, bc, center=CELL, prec=prec, green="hej2") as s:
        want = _device_solve(s, f, dt)
        h_in = _host(f, dt, pin_in)
        h_out = _host(np.zeros(shape), dt, pin_out)
        assert F.flups_host_mapped(h_in) == pin_in
        assert F.flups_host_mapped(h_out) == pin_out
        s.solve_host(h_out, h_in)
        assert s.check() == 0
        assert np.array_equal(h_out.numpy(), want)
        assert np.array_equal(h_in.numpy(), f.astype(h_in.numpy().dtype))  # rhs untouched


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_host_solve_in_place(pinned):
    import torch
    shape = (16, 32, 32)
    f = np.random.default_rng(4).standard_normal(shape)
    with F.Solver((32, 32, 16), ((U, U), (U, U), (E, E)), center=CELL, prec=F.F64, green="hej4") as s:
        want = _device_solve(s, f, torch.float64)
        h = _host(f, torch.float64, pinned)
        s.solve_host(h, h)
        assert np.array_equal(h.numpy(), want)


def test_host_solve_biot_savart_pinned():
    import torch
    shape = (3, 16, 24, 32)
    f = np.random.default_rng(5).standard_normal(shape)
    bc = (((U, U), (U, U), (O, O)), ((U, U), (U, U), (O, O)), ((U, U), (U, U), (E, E)))
    with F.Solver((32, 24, 16), bc, center=CELL, prec=F.F64, green="hej2", op=F.BIOT_SAVART, ncomp=3) as s:
        want = _device_solve(s, f, torch.float64)
        h_in = _host(f, torch.float64, True)
        h_out = _host(np.zeros(shape), torch.float64, True)
        s.solve_host(h_out, h_in)
        assert np.array_equal(h_out.numpy(), want)


def test_host_mapped_refuses_pageable_and_out_of_range():
    import torch
    a = np.zeros(1 << 16)
    assert not F.flups_host_mapped(a)
    t = torch.zeros(1 << 16, dtype=torch.float64).pin_memory()
    assert F.flups_host_mapped(t)
    assert F.flups_host_mapped(t, 8)
    assert not F.flups_host_mapped(t, 0)
