"""The oracle Poisson solve: a plain, slow FP64 CPU statement of the FLUPS method.

This module is test infrastructure: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA path.

What it computes (Section "Methodology"):

1. For every direction, the right-hand side is extended to a periodic signal
   by the rule of its boundary conditions:
     * periodic: the N samples (node layout: f_N is unused, Section 2.1/2.2);
     * even/odd faces (Table 1 and Sections 2.2.1-2.2.4): explicit even or odd
       reflection about both faces; period 2L when both faces have the same
       parity, 4L otherwise;
     * unbounded on both faces (Section 2.3.1, Hockney-Eastwood doubling):
       the samples followed by zeros up to period 2L (node layout: N+1 values
       then N-1 zeros, the Green's function symmetrised about j = N);
     * semi-unbounded (Section 2.3.2): zero padding to 2L on the unbounded
       side, then the even or odd reflection about the symmetric face
       (period 4L).
2. The Green's function is either a function of the continuous wavenumber of
   each extended mode (spectral directions) or is sampled in real space at
   the offsets m*h, m = min(p, P - p), of the extended period P and Fourier
   transformed (unbounded and semi-unbounded directions), times h per such
   direction.
3. u = G * f as a pointwise product in Fourier space (eq. poisson), computed
   with one full complex FFT over the extended box, then restricted to the
   original samples.  Node-centred boundary values are then set as the paper
   states: periodic phi_N := phi_0; an odd face holds 0.

The Biot-Savart variant (``biot_savart``, Section "Biot-Savart solver") takes
the curl in Fourier space on the extended signals with the spectral symbol or
the finite-difference symbols of orders 2, 4 and 6; the tests pin those
against real-space central-difference stencils and their convergence orders.

Everything is FP64.  Arrays are indexed [z, y, x] (x fastest, C order);
direction d = 0, 1, 2 (x, y, z) is numpy axis 2 - d.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import green as _green

EVEN, ODD, PER, UNB = 0, 1, 3, 4
CELL, NODE = 0, 1

SYMMETRIC = ("EE", "EO", "OE", "OO")
SEMI = ("EU", "OU", "UE", "UO")


def direction_type(left: int, right: int) -> str:
    """Classify one direction from its two face conditions (Section 1, the 4 categories)."""
    if PER in (left, right):
        if left != right:
            raise ValueError("a periodic condition must hold on both faces")
        return "PER"
    for b in (left, right):
        if b not in (EVEN, ODD, UNB):
            raise ValueError(f"unknown boundary condition {b}")
    if left == UNB and right == UNB:
        return "UNB"
    c = {EVEN: "E", ODD: "O", UNB: "U"}
    return c[left] + c[right]


def cost_class(t: str) -> int:
    """Transform cost class (Section 1): symmetric 1, semi-unbounded 2, periodic 3, unbounded 4."""
    if t in SYMMETRIC:
        return 1
    if t in SEMI:
        return 2
    if t == "PER":
        return 3
    return 4


def direction_order(types) -> list:
    """Directions sorted by cost class, ties kept in x, y, z order (Section 1)."""
    return sorted(range(3), key=lambda d: (cost_class(types[d]), d))


def n_cells(n_data: int, t: str, center: int) -> int:
    """N (cells) of a direction from its number of data values."""
    return n_data if center == CELL else n_data - 1


# ---------------------------------------------------------------------------
# 1D extension along axis 0 and restriction back.
# ---------------------------------------------------------------------------
def _cat(parts):
    return np.concatenate(parts, axis=0)


def extend(f: np.ndarray, t: str, center: int) -> np.ndarray:
    """Periodic extension of f along axis 0 (see the module docstring, step 1)."""
    if t in ("UE", "UO"):
        return extend(f[::-1], t[::-1], center)
    n = f.shape[0]
    z = np.zeros_like
    if center == CELL:
        N = n
        if t == "PER":
            return f.copy()
        if t == "UNB":
            return _cat([f, z(f)])
        if t == "EE":
            return _cat([f, f[::-1]])
        if t == "OO":
            return _cat([f, -f[::-1]])
        if t == "EO":  # even about x = 0, odd about x = L -> antiperiodic with 2L
            half = _cat([f, -f[::-1]])
            return _cat([half, -half])
        if t == "OE":
            half = _cat([f, f[::-1]])
            return _cat([half, -half])
        if t == "EU":  # pad to 2L, then even reflection about x = 0 (period 4L)
            g = _cat([f, z(f)])
            return _cat([g, g[::-1]])
        if t == "OU":
            g = _cat([f, z(f)])
            return _cat([g, -g[::-1]])
    else:
        N = n - 1
        if t == "PER":
            return f[:N].copy()
        if t == "UNB":
            return _cat([f, np.zeros((N - 1,) + f.shape[1:])])
        g = f.copy()
        if t == "EE":
            return _cat([g, g[N - 1:0:-1]])
        if t == "OO":
            g[0] = 0.0
            g[N] = 0.0
            return _cat([g, -g[N - 1:0:-1]])
        if t == "OE":  # odd about node 0, even about node N, period 4N
            g[0] = 0.0
            half = _cat([g, g[N - 1:0:-1]])
            return _cat([half, -half])
        if t == "EO":
            g[N] = 0.0
            half = _cat([g, -g[N - 1:0:-1]])
            return _cat([half, -half])
        if t in ("EU", "OU"):  # pad to 2N cells (nodes 0..2N), then node EE or OO on 2N
            gp = _cat([g, np.zeros((N,) + f.shape[1:])])
            M = 2 * N
            if t == "EU":
                return _cat([gp, gp[M - 1:0:-1]])
            gp[0] = 0.0
            gp[M] = 0.0
            return _cat([gp, -gp[M - 1:0:-1]])
    raise ValueError(f"unknown direction type {t}")


def restrict(e: np.ndarray, n_data: int, t: str, center: int) -> np.ndarray:
    """Original samples from the extended signal, with the node-centred boundary values."""
    if center == CELL:
        out = e[:n_data]
        return out[::-1].copy() if t in ("UE", "UO") else out.copy()
    N = n_data - 1
    if t == "PER":
        return _cat([e[:N], e[:1]])
    out = e[:n_data].copy()
    if t in ("UE", "UO"):
        out = out[::-1].copy()
    left_odd = t[0] == "O"
    right_odd = t[1] == "O"
    if left_odd:
        out[0] = 0.0
    if right_odd:
        out[N] = 0.0
    return out


def extended_length(n_data: int, t: str, center: int) -> int:
    N = n_cells(n_data, t, center)
    if t == "PER":
        return N
    if t in ("UNB", "EE", "OO"):
        return 2 * N
    return 4 * N  # EO, OE and the semi-unbounded directions


# ---------------------------------------------------------------------------
# The solve.
# ---------------------------------------------------------------------------
@dataclass
class Problem:
    bc: tuple            # ((xl, xr), (yl, yr), (zl, zr))
    h: tuple             # (hx, hy, hz)
    center: int = CELL
    kernel: str = "spectral"
    eps_over_h: float = 2.0

    def types(self):
        return [direction_type(*self.bc[d]) for d in range(3)]

    @property
    def eps(self) -> float:
        return self.eps_over_h * max(self.h)


# The complex FFT the solve uses as a library step: numpy's (one thread) unless
# set_fft_workers asked for scipy.fft with several worker threads.  Both compute
# the same unnormalised DFT; only the library call changes, none of the method's
# arithmetic.
_FFT_WORKERS = 1


def set_fft_workers(n: int) -> int:
    """Use scipy.fft with n worker threads for the oracle's FFTs (n <= 1: numpy, one thread).
    Returns the number of threads the FFTs will use."""
    global _FFT_WORKERS
    n = int(n)
    if n > 1:
        try:
            import scipy.fft  # noqa: F401
        except ImportError:
            n = 1
    _FFT_WORKERS = max(1, n)
    return _FFT_WORKERS


def _fftn(a, axes=None):
    if _FFT_WORKERS > 1:
        import scipy.fft
        return scipy.fft.fftn(a, axes=axes, workers=_FFT_WORKERS)
    return np.fft.fftn(a, axes=axes)


def _ifftn(a):
    if _FFT_WORKERS > 1:
        import scipy.fft
        return scipy.fft.ifftn(a, workers=_FFT_WORKERS)
    return np.fft.ifftn(a)


def _wavenumbers(P: int, h: float) -> np.ndarray:
    """Continuous wavenumber of each mode of a P-periodic extension (signed)."""
    p = np.arange(P)
    m = np.where(p <= P // 2, p, p - P)
    return 2.0 * math.pi * m / (P * h)


def _offsets(P: int, h: float) -> np.ndarray:
    """Real-space distance of each sample of the P-periodic symmetrised Green's function."""
    p = np.arange(P)
    return np.minimum(p, P - p) * h


def green_spectrum(prob: Problem, shape_ext) -> np.ndarray:
    """G^ on the full extended box (shape [Pz, Py, Px]), real, FP64."""
    types = prob.types()
    P = [shape_ext[2 - d] for d in range(3)]
    unb = [d for d in range(3) if types[d] == "UNB" or types[d] in SEMI]
    spec = [d for d in range(3) if d not in unb]

    def bcast(vec, d):
        shp = [1, 1, 1]
        shp[2 - d] = vec.size
        return vec.reshape(shp)

    if not unb:
        kd = [bcast(_wavenumbers(P[d], prob.h[d]), d) for d in range(3)]
        k2 = kd[0] ** 2 + kd[1] ** 2 + kd[2] ** 2
        k2, *kb = np.broadcast_arrays(k2, *kd)
        return _green.spectral_kernel(prob.kernel, k2, prob.eps, kdir=kb, h=prob.h)

    du = len(unb)
    k2 = np.zeros([1, 1, 1])
    for d in spec:
        k2 = k2 + bcast(_wavenumbers(P[d], prob.h[d]), d) ** 2
    r2 = np.zeros([1, 1, 1])
    for d in unb:
        r2 = r2 + bcast(_offsets(P[d], prob.h[d]), d) ** 2
    k2, r2 = np.broadcast_arrays(k2, r2)
    kmag = np.sqrt(k2)
    r = np.sqrt(r2)
    if prob.kernel in ("hej2", "hej4", "hej6", "hej8", "hej10"):
        g = _green.hej_mixed(int(prob.kernel[3:]) // 2, du, kmag, r, prob.eps)
    elif prob.kernel == "hej0" and du == 3:
        g = _green.hej0_3d(r, max(prob.h))
    elif prob.kernel == "lgf2" and du == 3:
        # evaluate on the folded offsets 0..P_d/2, then unfold (the samples are even in every direction)
        off = [np.minimum(np.arange(P[d]), P[d] - np.arange(P[d])) for d in range(3)]
        fold = [bcast(np.arange(P[d] // 2 + 1), d) for d in range(3)]
        fold = np.broadcast_arrays(*fold)
        gf = _green.lgf_3d(fold[0], fold[1], fold[2], prob.h)
        g = gf[np.ix_(off[2], off[1], off[0])]
    else:
        raise ValueError(f"kernel {prob.kernel!r} with {du} unbounded direction(s) is not in the oracle")
    axes = tuple(2 - d for d in unb)
    vol = float(np.prod([prob.h[d] for d in unb]))
    return (vol * _fftn(g, axes=axes)).real


def solve(f: np.ndarray, prob: Problem) -> np.ndarray:
    """phi with lap(phi) = f (eq. poisson), f indexed [z, y, x]; FP64."""
    f = np.asarray(f, dtype=np.float64)
    types = prob.types()
    e = f
    for d in range(3):
        ax = 2 - d
        e = np.moveaxis(extend(np.moveaxis(e, ax, 0), types[d], prob.center), 0, ax)
    G = green_spectrum(prob, e.shape)
    phi_e = _ifftn(G * _fftn(e)).real
    out = phi_e
    for d in range(3):
        ax = 2 - d
        out = np.moveaxis(restrict(np.moveaxis(out, ax, 0), f.shape[ax], types[d], prob.center), 0, ax)
    return np.ascontiguousarray(out)


# ---------------------------------------------------------------------------
# Biot-Savart: lap(u) = curl(f) (Section "Application: the Biot-Savart solver").
# ---------------------------------------------------------------------------
def curl_bc(bc_f):
    """Face conditions of each velocity component from those of the vorticity.

    bc_f[c][d] = (left, right) for component c of f.  Differentiation along d
    swaps even and odd in d; periodic and unbounded faces are kept.  Component
    c of curl(f) is d_{c+1} f_{c+2} - d_{c+2} f_{c+1}; its condition along d is
    that of f_{c+2} along d with the swap when d = c+1 (and, consistently, that
    of f_{c+1} with the swap when d = c+2).
    """
    def swap(b):
        return {EVEN: ODD, ODD: EVEN}.get(b, b)

    out = []
    for c in range(3):
        a, b = (c + 1) % 3, (c + 2) % 3
        comp = []
        for d in range(3):
            l, r = bc_f[b][d]
            if d == a:
                l, r = swap(l), swap(r)
            comp.append((l, r))
        out.append(tuple(comp))
    return tuple(out)


def biot_savart(f3: np.ndarray, bc_f, h, center=CELL, kernel="spectral", eps_over_h=2.0, diff="spectral"):
    """u with lap(u) = curl(f), f3 indexed [c, z, y, x]; spectral derivative i*k on the
    extended signals (the finite-difference symbols of the paper are selected with diff="fd2"/"fd4"/"fd6")."""
    f3 = np.asarray(f3, dtype=np.float64)
    bc_u = curl_bc(bc_f)
    shp = f3.shape[1:]
    ext = []
    for c in range(3):
        types = [direction_type(*bc_f[c][d]) for d in range(3)]
        e = f3[c]
        for d in range(3):
            ax = 2 - d
            e = np.moveaxis(extend(np.moveaxis(e, ax, 0), types[d], center), 0, ax)
        ext.append(e)
    if any(x.shape != ext[0].shape for x in ext):
        raise ValueError("components extend to different periods")
    Pshape = ext[0].shape
    F = [_fftn(x) for x in ext]
    # the derivative symbols act on the extended signals (real, Hermitian spectra)
    ik = []
    for d in range(3):
        P = Pshape[2 - d]
        kk = _wavenumbers(P, h[d])
        if diff == "spectral":
            sym = kk
        elif diff == "fd2":
            sym = np.sin(kk * h[d]) / h[d]
        elif diff == "fd4":
            sym = (4.0 / 3.0 * np.sin(kk * h[d]) - 1.0 / 6.0 * np.sin(2 * kk * h[d])) / h[d]
        elif diff == "fd6":
            sym = (1.5 * np.sin(kk * h[d]) - 0.3 * np.sin(2 * kk * h[d]) + np.sin(3 * kk * h[d]) / 30.0) / h[d]
        else:
            raise ValueError(diff)
        if P % 2 == 0:
            sym = sym.copy()
            sym[P // 2] = 0.0  # odd symbol: the Nyquist mode of a real signal has no derivative
        shp3 = [1, 1, 1]
        shp3[2 - d] = P
        ik.append(1j * sym.reshape(shp3))
    # Green's function: the same on all components (it depends on the BC kind, not parity)
    prob0 = Problem(bc=bc_u[0], h=h, center=center, kernel=kernel, eps_over_h=eps_over_h)
    G = green_spectrum(prob0, Pshape)
    out = np.empty((3,) + shp)
    for c in range(3):
        a, b = (c + 1) % 3, (c + 2) % 3
        curl = ik[a] * F[b] - ik[b] * F[a]
        u_e = _ifftn(G * curl).real
        types_u = [direction_type(*bc_u[c][d]) for d in range(3)]
        o = u_e
        for d in range(3):
            ax = 2 - d
            o = np.moveaxis(restrict(np.moveaxis(o, ax, 0), shp[ax], types_u[d], center), 0, ax)
        out[c] = o
    return out
