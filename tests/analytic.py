"""Analytic reference solutions of the paper's validation cases (test helpers).

Appendix "Analytical expressions used for the validation": phi_ref is a product
of 1D functions and f = lap(phi_ref) is formed analytically (Section
"Validation").  These are expected values taken from the paper, not results of
either implementation.
"""
import math

import numpy as np


def bump(x, c, L=1.0):
    """exp(10 (1 - 1/(1 - ((2x - c L)/L)^2))) inside its support, 0 outside, and d2/dx2."""
    u = (2.0 * x - c * L) / L
    val = np.zeros_like(x, dtype=np.float64)
    d2 = np.zeros_like(x, dtype=np.float64)
    m = np.abs(u) < 1.0
    uu = u[m]
    q = 1.0 - uu * uu
    g = 10.0 * (1.0 - 1.0 / q)
    gp = -20.0 * uu / q ** 2
    gpp = -10.0 * (2.0 / q ** 2 + 8.0 * uu * uu / q ** 3)
    X = np.exp(g)
    val[m] = X
    d2[m] = X * (gp * gp + gpp) * (2.0 / L) ** 2
    return val, d2


def separable(X, Y, Z):
    """phi = X(x) Y(y) Z(z) and f = X''YZ + XY''Z + XYZ'' on [z, y, x] arrays."""
    (x0, x2), (y0, y2), (z0, z2) = X, Y, Z
    phi = z0[:, None, None] * y0[None, :, None] * x0[None, None, :]
    f = (z0[:, None, None] * y0[None, :, None] * x2[None, None, :]
         + z0[:, None, None] * y2[None, :, None] * x0[None, None, :]
         + z2[:, None, None] * y0[None, :, None] * x0[None, None, :])
    return phi, f


def case_symmetric_periodic(N, L=1.0):
    """phi = cos(pi x/L) sin(5 pi y/(2L)) sin(8 pi z/L), node-centred, x EE, y OE, z periodic."""
    x = np.arange(N + 1) * (L / N)
    X = (np.cos(math.pi * x / L), -(math.pi / L) ** 2 * np.cos(math.pi * x / L))
    ky = 2.5 * math.pi / L
    Y = (np.sin(ky * x), -ky * ky * np.sin(ky * x))
    kz = 8.0 * math.pi / L
    Z = (np.sin(kz * x), -kz * kz * np.sin(kz * x))
    return separable(X, Y, Z)


def case_unbounded(N, L=1.0):
    x = np.arange(N + 1) * (L / N)
    b = bump(x, 1.0, L)
    return separable(b, b, b)


def case_semi_unbounded(N, L=1.0):
    x = np.arange(N + 1) * (L / N)
    a1, a2 = bump(x, 1.4, L), bump(x, 2.6, L)
    X = (a1[0] + a2[0], a1[1] + a2[1])
    Y = bump(x, 1.0, L)
    b1, b2 = bump(x, 0.6, L), bump(x, -0.6, L)
    Z = (b1[0] - b2[0], b1[1] - b2[1])
    return separable(X, Y, Z)


def gaussian_potential(r, sigma):
    """Potential of a unit-mass Gaussian of width sigma: -erf(r/(sqrt2 sigma))/(4 pi r)."""
    from scipy.special import erf
    r = np.asarray(r, dtype=np.float64)
    out = np.full_like(r, -1.0 / ((2.0 * math.pi) ** 1.5 * sigma))
    nz = r > 0
    out[nz] = -erf(r[nz] / (math.sqrt(2.0) * sigma)) / (4.0 * math.pi * r[nz])
    return out


def vortex_tube(N, nz, R, L=1.0):
    """The paper's Biot-Savart validation (Section "Application: the Biot-Savart solver"): a compact
    vortex tube along z centred at (L/2, L/2), radius R, node-centred N + 1 points in x and y and
    nz + 1 in z.  Returns (f, u): f = (0, 0, -w(r)) with w(r) = (1/2 pi)(2/R^2)(1/E2(1))
    exp(-1/(1 - (r/R)^2)) inside R (the field handed to the solver, lap(u) = curl f) and the
    analytical velocity u = (-sin(theta) u_t, cos(theta) u_t, 0) with
    u_t(r) = (1/(2 pi r)) [1 - (1 - (r/R)^2) E2(1/(1 - (r/R)^2)) / E2(1)] inside R, 1/(2 pi r) outside.
    Arrays are [c, z, y, x]."""
    from scipy.special import expn
    x = np.arange(N + 1) * (L / N) - 0.5 * L
    X, Y = np.meshgrid(x, x, indexing="xy")        # [y, x]
    r = np.sqrt(X * X + Y * Y)
    q = (r / R) ** 2
    inside = q < 1.0
    e21 = expn(2, 1.0)
    w = np.zeros_like(r)
    w[inside] = (1.0 / (2 * math.pi)) * (2.0 / (R * R)) / e21 * np.exp(-1.0 / (1.0 - q[inside]))
    ut = np.zeros_like(r)
    rr = np.where(r > 0, r, 1.0)
    ut_out = 1.0 / (2 * math.pi * rr)
    s = np.where(inside, 1.0 - q, 1.0)
    ut_in = ut_out * (1.0 - s * expn(2, 1.0 / s) / e21)
    ut = np.where(inside, ut_in, ut_out)
    ut = np.where(r > 0, ut, 0.0)
    ux = -Y / rr * ut
    uy = X / rr * ut
    f = np.zeros((3, nz + 1, N + 1, N + 1))
    f[2] = -w[None, :, :]
    u = np.zeros_like(f)
    u[0] = ux[None]
    u[1] = uy[None]
    return f, u
