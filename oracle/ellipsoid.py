"""Semi-analytic potential of a homogeneous ellipsoid (validation of §5).

TEST INFRASTRUCTURE: the reference solution that the ellipsoid validation
compares the solver with.  Only tests/ may import it; it shares no code with
the library.

§5 writes the potential of a homogeneous ellipsoid of density rho0 and
semi-axes a, b, c (Chandrasekhar 1969) as

    Phi(x) = pi G rho0 a b c (A x^2 + B y^2 + C z^2 - D),

with A, B, C, D integrals over u from u0 to infinity of
[(a^2+u)(b^2+u)(c^2+u)]^(-1/2) times 1/(a^2+u), 1/(b^2+u), 1/(c^2+u) and 1,
and u0 = 0 inside, else the positive root of
x^2/(a^2+u) + y^2/(b^2+u) + z^2/(c^2+u) = 1.

Shifting u by u0 turns them into Carlson's symmetric integrals
    R_F(x, y, z) = 1/2 int_0^inf dt [(t+x)(t+y)(t+z)]^(-1/2),
    R_D(x, y, z) = 3/2 int_0^inf dt [(t+x)(t+y)]^(-1/2) (t+z)^(-3/2):
    D = 2 R_F(a'^2, b'^2, c'^2),  A = 2/3 R_D(b'^2, c'^2, a'^2),
    B = 2/3 R_D(a'^2, c'^2, b'^2), C = 2/3 R_D(a'^2, b'^2, c'^2),
with a'^2 = a^2 + u0 and so on.  R_F and R_D are evaluated by Carlson's
duplication method (B. C. Carlson, "Numerical computation of real or complex
elliptic integrals", Numer. Algorithms 10 (1995) 13-26): repeated
duplication x -> (x + lambda) / 4 until the arguments agree to about 1e-3,
then the fifth-order Taylor series in the elementary symmetric functions of
the relative deviations.  u0 is bracketed in [0, r^2] and found by bisection
followed by Newton steps.
"""

from __future__ import annotations

import math

import numpy as np


def carlson_rf(x, y, z):
    """R_F(x, y, z) for x, y, z >= 0, at most one of them zero (vectorised)."""
    x, y, z = (np.array(v, dtype=np.float64, copy=True) for v in np.broadcast_arrays(x, y, z))
    for _ in range(40):
        A = (x + y + z) / 3.0
        dev = np.maximum(np.maximum(np.abs(A - x), np.abs(A - y)), np.abs(A - z)) / A
        if np.all(dev < 1e-3):
            break
        sx, sy, sz = np.sqrt(x), np.sqrt(y), np.sqrt(z)
        lam = sx * sy + sy * sz + sz * sx
        x, y, z = (x + lam) / 4.0, (y + lam) / 4.0, (z + lam) / 4.0
    A = (x + y + z) / 3.0
    X, Y = (A - x) / A, (A - y) / A
    Z = -(X + Y)
    E2 = X * Y - Z * Z
    E3 = X * Y * Z
    return (1.0 - E2 / 10.0 + E3 / 14.0 + E2 * E2 / 24.0 - 3.0 * E2 * E3 / 44.0) / np.sqrt(A)


def carlson_rd(x, y, z):
    """R_D(x, y, z) for x, y >= 0 (not both zero) and z > 0 (vectorised)."""
    x, y, z = (np.array(v, dtype=np.float64, copy=True) for v in np.broadcast_arrays(x, y, z))
    acc = np.zeros_like(x)
    scale = np.ones_like(x)                 # 4^-m
    for _ in range(40):
        A = (x + y + 3.0 * z) / 5.0
        dev = np.maximum(np.maximum(np.abs(A - x), np.abs(A - y)), np.abs(A - z)) / A
        if np.all(dev < 1e-3):
            break
        sx, sy, sz = np.sqrt(x), np.sqrt(y), np.sqrt(z)
        lam = sx * sy + sy * sz + sz * sx
        acc += scale / (sz * (z + lam))
        scale = scale / 4.0
        x, y, z = (x + lam) / 4.0, (y + lam) / 4.0, (z + lam) / 4.0
    A = (x + y + 3.0 * z) / 5.0
    X, Y = (A - x) / A, (A - y) / A
    Z = -(X + Y) / 3.0
    XY = X * Y
    E2 = XY - 6.0 * Z * Z
    E3 = (3.0 * XY - 8.0 * Z * Z) * Z
    E4 = 3.0 * (XY - Z * Z) * Z * Z
    E5 = XY * Z ** 3
    series = (1.0 - 3.0 * E2 / 14.0 + E3 / 6.0 + 9.0 * E2 * E2 / 88.0 - 3.0 * E4 / 22.0
              - 9.0 * E2 * E3 / 52.0 + 3.0 * E5 / 26.0)
    return scale * series / (A * np.sqrt(A)) + 3.0 * acc


def confocal_root(x, y, z, a, b, c):
    """u0 of §5: 0 where (x/a)^2 + (y/b)^2 + (z/c)^2 <= 1, else the positive
    root of x^2/(a^2+u) + y^2/(b^2+u) + z^2/(c^2+u) = 1 (the left side falls
    monotonically in u and is <= 1 at u = r^2)."""
    x2, y2, z2 = x * x, y * y, z * z
    a2, b2, c2 = a * a, b * b, c * c
    f = lambda u: x2 / (a2 + u) + y2 / (b2 + u) + z2 / (c2 + u) - 1.0
    outside = f(0.0) > 0.0
    lo = np.zeros_like(x2)
    hi = np.where(outside, x2 + y2 + z2, 0.0)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        pos = f(mid) > 0.0
        lo = np.where(pos, mid, lo)
        hi = np.where(pos, hi, mid)
    u = 0.5 * (lo + hi)
    for _ in range(2):   # Newton polish; f' = -sum x_i^2 / (a_i^2 + u)^2 < 0 outside
        fp = -(x2 / (a2 + u) ** 2 + y2 / (b2 + u) ** 2 + z2 / (c2 + u) ** 2)
        step = np.where(outside, f(u) / np.where(outside, fp, -1.0), 0.0)
        u = np.clip(u - step, lo, hi)
    return np.where(outside, u, 0.0)


def ellipsoid_potential(x, y, z, axes, rho0=1.0, G=1.0):
    """Phi at points given in the ellipsoid's frame (arrays of one shape)."""
    a, b, c = (float(v) for v in axes)
    x, y, z = (np.asarray(v, dtype=np.float64) for v in (x, y, z))
    u = confocal_root(x, y, z, a, b, c)
    A2, B2, C2 = a * a + u, b * b + u, c * c + u
    D = 2.0 * carlson_rf(A2, B2, C2)
    Ai = 2.0 / 3.0 * carlson_rd(B2, C2, A2)
    Bi = 2.0 / 3.0 * carlson_rd(A2, C2, B2)
    Ci = 2.0 / 3.0 * carlson_rd(A2, B2, C2)
    return math.pi * G * rho0 * a * b * c * (Ai * x * x + Bi * y * y + Ci * z * z - D)


def ellipsoid_potential_on_grid(r_out, units, axes, dphi=math.pi / 8, rho0=1.0, G=1.0, chunk=1 << 20):
    """Phi at radii r_out (the solver's r_n^+) and global-frame unit vectors
    units [3, ...] of the target cells; the ellipsoid frame is the global one
    turned by dphi about z (§5: x = r sin(theta) cos(phi + dphi), ...).
    Returns shape (n_r,) + units.shape[1:]."""
    r_out = np.asarray(r_out, dtype=np.float64)
    cd, sd = math.cos(dphi), math.sin(dphi)
    ux, uy, uz = (np.asarray(units[k], dtype=np.float64).reshape(-1) for k in range(3))
    ex, ey = cd * ux - sd * uy, sd * ux + cd * uy
    out = np.empty((r_out.size, ux.size))
    rows = max(1, chunk // max(1, ux.size))
    for i0 in range(0, r_out.size, rows):
        rr = r_out[i0:i0 + rows, None]
        out[i0:i0 + rows] = ellipsoid_potential(rr * ex[None], rr * ey[None], rr * uz[None], axes, rho0, G)
    return out.reshape((r_out.size,) + np.asarray(units[0]).shape)
