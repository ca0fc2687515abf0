"""Seeded synthetic right-hand sides for the solver's workloads.

This module only draws random numbers and samples analytic source fields; it
holds none of the solver's arithmetic, and both the CUDA path's callers and the
CPU oracle's callers use it.  Arrays are float64, indexed [z, y, x] (x fastest),
or [c, z, y, x] for vector fields.

The shapes and value distributions follow the paper's validation workloads
(Section "Validation": products of sines on spectral BCs, compact/Gaussian
blobs on unbounded BCs; Section "Application: the Biot-Savart solver": a
compact vorticity distribution) at the sizes of the benchmark configurations.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

CELL, NODE = 0, 1
EVEN, ODD, PER, UNB = 0, 1, 3, 4


def coords(n: int, L: float, center: int, n_cells: int | None = None) -> np.ndarray:
    """Sample positions: cell x_j = (j + 1/2) h, node x_j = j h, with h = L / n_cells."""
    if n_cells is None:
        n_cells = n if center == CELL else n - 1
    h = L / n_cells
    j = np.arange(n, dtype=np.float64)
    return (j + 0.5) * h if center == CELL else j * h


# ---------------------------------------------------------------------------
# Fully periodic sine products (periodic 32^3 FP64 and 1024^3 FP64 workloads).
# ---------------------------------------------------------------------------
def sine_modes(seed: int, nmodes: int = 4, kmax: int = 4):
    """nmodes (a, b, c, A): integer wavenumbers in [1, kmax], amplitudes U(-1, 1)."""
    rng = np.random.default_rng(seed)
    abc = rng.integers(1, kmax + 1, size=(nmodes, 3))
    amp = rng.uniform(-1.0, 1.0, size=nmodes)
    return [(int(a), int(b), int(c), float(A)) for (a, b, c), A in zip(abc, amp)]


def periodic_sines(n, modes, L=1.0, center=CELL, dtype=np.float64):
    """f = sum_m A_m sin(2 pi a x/L) sin(2 pi b y/L) sin(2 pi c z/L) on an n[0] x n[1] x n[2] grid."""
    nx, ny, nz = n
    x = coords(nx, L, center)
    y = coords(ny, L, center)
    z = coords(nz, L, center)
    f = np.zeros((nz, ny, nx), dtype=dtype)
    for a, b, c, A in modes:
        sx = np.sin(2 * math.pi * a * x / L).astype(dtype)
        sy = np.sin(2 * math.pi * b * y / L).astype(dtype)
        sz = np.sin(2 * math.pi * c * z / L).astype(dtype)
        f += dtype(A) * sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    return f


def periodic_sines_torch(n, modes, device, dtype, L=1.0, center=CELL):
    """The same field built on a device with torch (for the 1024^3 workload)."""
    import torch
    nx, ny, nz = n
    x = torch.as_tensor(coords(nx, L, center), device=device, dtype=torch.float64)
    y = torch.as_tensor(coords(ny, L, center), device=device, dtype=torch.float64)
    z = torch.as_tensor(coords(nz, L, center), device=device, dtype=torch.float64)
    f = torch.zeros((nz, ny, nx), device=device, dtype=dtype)
    for a, b, c, A in modes:
        sx = torch.sin(2 * math.pi * a * x / L).to(dtype)
        sy = torch.sin(2 * math.pi * b * y / L).to(dtype)
        sz = torch.sin(2 * math.pi * c * z / L).to(dtype)
        f += A * sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    return f


def periodic_sines_planes(n, modes, zidx, L=1.0, center=CELL):
    """The same field restricted to the z-planes zidx (for sampled checks at large n)."""
    nx, ny, nz = n
    x = coords(nx, L, center)
    y = coords(ny, L, center)
    z = coords(nz, L, center)[np.asarray(zidx)]
    f = np.zeros((len(z), ny, nx))
    for a, b, c, A in modes:
        f += A * np.sin(2 * math.pi * c * z / L)[:, None, None] * np.sin(2 * math.pi * b * y / L)[None, :, None] \
            * np.sin(2 * math.pi * a * x / L)[None, None, :]
    return f


# ---------------------------------------------------------------------------
# Gaussian blob (unbounded 128^3 and 512^3 workloads).
# ---------------------------------------------------------------------------
def blob_center(seed: int, jitter: float = 1e-3, base=(0.5, 0.5, 0.5)):
    rng = np.random.default_rng(seed)
    return tuple(float(b + d) for b, d in zip(base, rng.uniform(-jitter, jitter, size=3)))


def gaussian_blob(n, sigma, center_xyz, L=(1.0, 1.0, 1.0), center=CELL, dtype=np.float64):
    """Unit-mass Gaussian (2 pi sigma^2)^{-3/2} exp(-r^2 / (2 sigma^2))."""
    nx, ny, nz = n
    x = coords(nx, L[0], center) - center_xyz[0]
    y = coords(ny, L[1], center) - center_xyz[1]
    z = coords(nz, L[2], center) - center_xyz[2]
    c = (2 * math.pi * sigma * sigma) ** -1.5
    gx = np.exp(-x * x / (2 * sigma * sigma))
    gy = np.exp(-y * y / (2 * sigma * sigma))
    gz = np.exp(-z * z / (2 * sigma * sigma))
    return (c * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]).astype(dtype)


# ---------------------------------------------------------------------------
# Mixed-BC workload: node-centred 257 x 256 x 257, x symmetric, y periodic
# (stored without the duplicate node), z unbounded.
# ---------------------------------------------------------------------------
def mixed_blob_modes(n=(257, 256, 257), h=1.0 / 256, sigma=0.08, seed=3, nmodes=4, center=(0.5, 0.5, 0.5)):
    """Gaussian blob plus nmodes seeded terms A sin(2 pi b y) g(x) g(z)."""
    nx, ny, nz = n
    x = np.arange(nx) * h - center[0]
    y = np.arange(ny) * h
    z = np.arange(nz) * h - center[2]
    gx = np.exp(-x * x / (2 * sigma * sigma))
    gz = np.exp(-z * z / (2 * sigma * sigma))
    yc = y - center[1]
    gy = np.exp(-yc * yc / (2 * sigma * sigma))
    c = (2 * math.pi * sigma * sigma) ** -1.5
    f = c * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    rng = np.random.default_rng(seed)
    b = rng.integers(1, 5, size=nmodes)
    A = rng.uniform(-1.0, 1.0, size=nmodes)
    for bb, AA in zip(b, A):
        f = f + AA * c * gz[:, None, None] * np.sin(2 * math.pi * bb * y)[None, :, None] * gx[None, None, :]
    return f


# ---------------------------------------------------------------------------
# Vorticity: Gaussian vortex ring (Biot-Savart requests of the served stream).
# ---------------------------------------------------------------------------
def vortex_ring(n, R0=0.25, sigma=0.05, gamma=1.0, L=1.0, center=CELL, axis_center=(0.5, 0.5, 0.5)):
    """omega = gamma/(2 pi sigma^2) exp(-d^2/(2 sigma^2)) e_theta, ring of radius R0 about z."""
    nx, ny, nz = n
    x = coords(nx, L, center) - axis_center[0]
    y = coords(ny, L, center) - axis_center[1]
    z = coords(nz, L, center) - axis_center[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    rho = np.sqrt(X * X + Y * Y)
    d2 = (rho - R0) ** 2 + Z * Z
    w = gamma / (2 * math.pi * sigma * sigma) * np.exp(-d2 / (2 * sigma * sigma))
    rs = np.where(rho > 0, rho, 1.0)
    out = np.zeros((3,) + X.shape)
    out[0] = -w * Y / rs
    out[1] = w * X / rs
    return out


# ---------------------------------------------------------------------------
# The served request stream.
# ---------------------------------------------------------------------------
@dataclass
class Request:
    rid: int
    arrival_s: float
    n: tuple
    bc: tuple            # ((xl, xr), (yl, yr), (zl, zr)) of the (first) component
    op: int              # 0 Poisson, 1 Biot-Savart
    prec: int            # 0 FP32, 1 FP64
    kernel: int          # green kernel enum of the C ABI
    seed: int = 0
    extra: dict = field(default_factory=dict)


SERVED_SIZES = (32, 64, 96, 128, 192, 256)


def _draw_bc(rng):
    """One direction: periodic on both faces, or each face from {even, odd, unbounded}."""
    if rng.uniform() < 0.25:
        return (PER, PER)
    return (int(rng.choice([EVEN, ODD, UNB])), int(rng.choice([EVEN, ODD, UNB])))


def served_stream(nreq=4096, seed=4, rate_hz=1000.0, bs_frac=0.3, fp32_frac=0.5, sizes=SERVED_SIZES):
    """Seeded request list with Poisson arrivals at rate_hz (exponential gaps)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(nreq):
        t += float(rng.exponential(1.0 / rate_hz))
        nn = int(rng.choice(sizes))
        op = 1 if rng.uniform() < bs_frac else 0
        prec = 0 if rng.uniform() < fp32_frac else 1
        if op == 1:
            # Biot-Savart: the ring lies in the xy plane; x and y unbounded or periodic, z any
            bx = (UNB, UNB) if rng.uniform() < 0.7 else (PER, PER)
            bz = _draw_bc(rng)
            bc = (bx, bx, bz)
        else:
            bc = tuple(_draw_bc(rng) for _ in range(3))
        any_unb = any(UNB in b for b in bc)
        kernel = 2 if any_unb else 0   # HEJ2 when any face is unbounded, spectral otherwise
        reqs.append(Request(rid=i, arrival_s=t, n=(nn, nn, nn), bc=bc, op=op, prec=prec, kernel=kernel,
                            seed=int(rng.integers(0, 2**31 - 1))))
    return reqs


def request_rhs(req: Request) -> np.ndarray:
    """The right-hand side of a served request (cell-centred, L = 1).  It depends only on the
    request's class (size and operator), so one pinned input serves every request of a class."""
    if req.op == 1:
        return vortex_ring(req.n)
    rng = np.random.default_rng(1000 + req.n[0])
    c = tuple(float(v) for v in 0.5 + rng.uniform(-0.05, 0.05, size=3))
    return gaussian_blob(req.n, 0.1, c)
