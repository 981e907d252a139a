"""Seeded synthetic workloads: grid descriptors and cell-averaged densities.

This module holds no part of the solver's arithmetic.  It only builds the
grid parameters and the density arrays that both the CUDA library and the
CPU oracle receive, so that the two see identical inputs.

Densities are defined in a global Cartesian frame equal to the Yin frame.
A Yang cell's local Cartesian position (x, y, z) sits at (-x, z, y) in the
global frame (the Yin-Yang map, its own inverse).  Arrays are float64
[n_r][n_theta][n_phi] per patch, C-contiguous.

A full spherical polar grid (``GridSpec.polar``) has one patch covering
theta in [0, pi] and phi in [0, 2 pi) in the global frame; the density
functions then return (rho, None).
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class GridSpec:
    """Parameters of one Yin-Yang grid (both patches share them)."""
    name: str
    r_edges: np.ndarray      # n_r + 1 strictly increasing radii, r_edges[0] >= 0
    n_theta: int
    n_phi: int
    delta_theta: float       # buffer widths (radians)
    delta_phi: float
    lmax: int
    G: float = 1.0
    polar: bool = False      # one patch over the whole sphere (buffers unused)

    @property
    def n_r(self) -> int:
        return int(self.r_edges.size - 1)

    @property
    def n_ang(self) -> int:
        return self.n_theta * self.n_phi


def _patch_step(n_theta, n_phi, delta_theta, delta_phi):
    dth = (math.pi / 2 + 2 * delta_theta) / n_theta
    dph = (3 * math.pi / 2 + 2 * delta_phi) / n_phi
    return dth, dph


def angular_cell_edges(spec: GridSpec):
    """Cell edges in theta and phi of one patch (both patches share them)."""
    if spec.polar:
        return (math.pi / spec.n_theta * np.arange(spec.n_theta + 1),
                2 * math.pi / spec.n_phi * np.arange(spec.n_phi + 1))
    dth, dph = _patch_step(spec.n_theta, spec.n_phi, spec.delta_theta, spec.delta_phi)
    return (math.pi / 4 - spec.delta_theta + dth * np.arange(spec.n_theta + 1),
            -3 * math.pi / 4 - spec.delta_phi + dph * np.arange(spec.n_phi + 1))


def patches(spec: GridSpec):
    return ("yin",) if spec.polar else ("yin", "yang")


def tiny_grid() -> GridSpec:
    """32 log-spaced zones in [1e-3, 1], 16 x 48 cells per patch, a buffer of
    two cells in theta and in phi, l_max = 8.  With d = 2 cells the cell sizes
    solve n * d_cell = range + 4 d_cell: 7.5 deg in theta, 3 pi / 88 in phi."""
    n_t, n_p = 16, 48
    dth = (math.pi / 2) / (n_t - 4)
    dph = (3 * math.pi / 2) / (n_p - 4)
    return GridSpec("tiny", np.logspace(-3, 0, 33), n_t, n_p, 2 * dth, 2 * dph, 8)


def mid_grid() -> GridSpec:
    """200 log-spaced zones in [1e-3, 1], 2-degree cells (45 x 135), l_max = 15."""
    return GridSpec("mid", np.logspace(-3, 0, 201), 45, 135, 0.0, 0.0, 15)


def production_grid() -> GridSpec:
    """550 log-spaced zones in [1e-4, 1], 1-degree cells (90 x 270), l_max = 25."""
    return GridSpec("production", np.logspace(-4, 0, 551), 90, 270, 0.0, 0.0, 25)


def polar_grid(r_edges, n_theta, n_phi, lmax, name="polar", G=1.0) -> GridSpec:
    """Full spherical polar grid: theta_j^+- = (j, j+1) pi / n_theta,
    phi_k^+- = (k, k+1) 2 pi / n_phi."""
    return GridSpec(name, np.asarray(r_edges, dtype=np.float64), n_theta, n_phi, 0.0, 0.0, lmax, G, True)


def tiny_polar_grid() -> GridSpec:
    """32 log-spaced zones in [1e-3, 1], 16 x 32 cells (11.25 degrees), l_max = 8."""
    return polar_grid(np.logspace(-3, 0, 33), 16, 32, 8, "tiny_polar")


def mid_polar_grid() -> GridSpec:
    """200 log-spaced zones in [1e-3, 1], 2-degree cells (90 x 180), l_max = 15."""
    return polar_grid(np.logspace(-3, 0, 201), 90, 180, 15, "mid_polar")


GRIDS = {"tiny": tiny_grid, "mid": mid_grid, "production": production_grid,
         "tiny_polar": tiny_polar_grid, "mid_polar": mid_polar_grid}


def cell_centres(spec: GridSpec):
    """Cell-centre radius, angles and global-frame unit vectors of both patches.

    Returns r_c [n_r], and for each patch the unit vectors [3, n_theta, n_phi]
    of the cell-centre directions in the global (Yin) frame.
    """
    te, pe = angular_cell_edges(spec)
    th = 0.5 * (te[:-1] + te[1:])
    ph = 0.5 * (pe[:-1] + pe[1:])
    T, P = np.meshgrid(th, ph, indexing="ij")
    local = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)])
    r_c = 0.5 * (spec.r_edges[:-1] + spec.r_edges[1:])
    if spec.polar:
        return r_c, {"yin": local}
    yang_global = np.stack([-local[0], local[2], local[1]])
    return r_c, {"yin": local, "yang": yang_global}


# ---------------------------------------------------------------------------
# densities
# ---------------------------------------------------------------------------

def centred_sphere_density(spec: GridSpec, radius: float, rho0: float):
    """Cell averages of a uniform sphere about the origin: the exact fraction
    of each zone's volume inside ``radius`` (independent of angle)."""
    rm, rp = spec.r_edges[:-1], spec.r_edges[1:]
    inside = np.clip(np.minimum(rp, radius) ** 3 - rm ** 3, 0.0, None) / (rp ** 3 - rm ** 3)
    rho = rho0 * inside[:, None, None] * np.ones((1, spec.n_theta, spec.n_phi))
    return rho.copy(), (None if spec.polar else rho.copy())


def offcentre_sphere_density(spec: GridSpec, centre, radius: float, rho0: float, q: int = 4):
    """Cell averages of a uniform sphere of ``radius`` centred at ``centre``:
    the indicator averaged over a q x q x q Gauss-Legendre product rule in
    (r^3, cos theta, phi), which is uniform in volume within each cell."""
    c = np.asarray(centre, dtype=np.float64)
    g, gw = np.polynomial.legendre.leggauss(q)
    u = 0.5 * (g + 1.0)              # nodes on [0, 1]
    uw = 0.5 * gw                    # weights summing to 1
    th_e, ph_e = angular_cell_edges(spec)
    dph = ph_e[1] - ph_e[0]
    r3m, r3p = spec.r_edges[:-1] ** 3, spec.r_edges[1:] ** 3
    r_s = np.cbrt(r3m[:, None] + (r3p - r3m)[:, None] * u[None, :])              # [n_r, q]
    cm, cp = np.cos(th_e[:-1]), np.cos(th_e[1:])
    ct_s = cm[:, None] + (cp - cm)[:, None] * u[None, :]                           # [n_t, q]
    st_s = np.sqrt(np.clip(1.0 - ct_s ** 2, 0.0, None))
    ph_s = ph_e[:-1, None] + dph * u[None, :]                                      # [n_p, q]
    out = {"yang": None}
    for patch in patches(spec):
        # local unit vectors at sub-points: [3, n_t, q, n_p, q]
        x = st_s[:, :, None, None] * np.cos(ph_s)[None, None, :, :]
        y = st_s[:, :, None, None] * np.sin(ph_s)[None, None, :, :]
        z = np.broadcast_to(ct_s[:, :, None, None], x.shape)
        if patch == "yang":
            x, y, z = -x, z, y
        acc = np.zeros((spec.n_r, spec.n_theta, spec.n_phi))
        for a in range(q):
            rr = r_s[:, a][:, None, None, None, None]
            d2 = (rr * x - c[0]) ** 2 + (rr * y - c[1]) ** 2 + (rr * z - c[2]) ** 2
            ind = (d2 <= radius * radius).astype(np.float64)
            acc += uw[a] * np.einsum("itbkc,b,c->itk", ind, uw, uw)
        out[patch] = rho0 * acc
    return out["yin"], out["yang"]


def tiny_density(spec: GridSpec | None = None):
    """Uniform sphere R = 0.3, rho = 1 at the origin plus a sphere a = 0.1,
    rho = 5 at (0.2, 0.1, -0.15), superposed."""
    spec = spec or tiny_grid()
    a_yin, a_yang = centred_sphere_density(spec, 0.3, 1.0)
    b_yin, b_yang = offcentre_sphere_density(spec, (0.2, 0.1, -0.15), 0.1, 5.0)
    return a_yin + b_yin, (None if spec.polar else a_yang + b_yang)


def oblate_density(spec: GridSpec | None = None, seed: int = 1):
    """rho = (1 + (x^2 + y^2)/0.2^2 + z^2/0.15^2)^-2 (1 + 0.05 N(0,1)) at cell
    centres, noise drawn in the order (patch, shell, theta, phi)."""
    spec = spec or mid_grid()
    rng = np.random.default_rng(seed)
    r_c, units = cell_centres(spec)
    out = {"yang": None}
    for patch in patches(spec):
        u = units[patch]
        X = r_c[:, None, None] * u[0][None]
        Y = r_c[:, None, None] * u[1][None]
        Z = r_c[:, None, None] * u[2][None]
        base = (1.0 + (X ** 2 + Y ** 2) / 0.04 + Z ** 2 / 0.0225) ** -2
        noise = rng.standard_normal(base.shape)
        out[patch] = base * (1.0 + 0.05 * noise)
    return out["yin"], out["yang"]


# monomials x^a y^b z^c with 1 <= a + b + c <= 4: on the unit sphere they span
# the same functions as the real harmonics of degree 0..4 minus the constant
_MONOMIALS = [(a, b, d - a - b) for d in range(1, 5) for a in range(d + 1) for b in range(d + 1 - a)]


def pns_density(spec: GridSpec | None = None, seed: int = 2, eps_scale: float = 0.02):
    """rho = [exp(-r/0.02) + 1e-4 r^-2.5] (1 + sum_i eps_i x^a y^b z^c) at cell
    centres (unit-vector components), eps_i ~ N(0, eps_scale^2) drawn in the
    order of the monomial list; a band-limited (degree <= 4) angular
    perturbation of a proto-neutron-star-like profile."""
    spec = spec or production_grid()
    rng = np.random.default_rng(seed)
    eps = rng.normal(0.0, eps_scale, size=len(_MONOMIALS))
    r_c, units = cell_centres(spec)
    radial = np.exp(-r_c / 0.02) + 1e-4 * r_c ** -2.5
    out = {"yang": None}
    for patch in patches(spec):
        u = units[patch]
        ang = np.ones(u.shape[1:])
        for e, (a, b, c) in zip(eps, _MONOMIALS):
            ang = ang + e * u[0] ** a * u[1] ** b * u[2] ** c
        out[patch] = radial[:, None, None] * ang[None]
    return out["yin"], out["yang"]


def ellipsoid_density(spec: GridSpec, axes, rho0: float = 1.0, dphi: float = math.pi / 8, q: int = 4):
    """Cell averages of the homogeneous ellipsoid (x/a)^2 + (y/b)^2 + (z/c)^2 <= 1
    (density rho0 inside), whose frame is the global one turned by dphi about z:
    a point at global angles (theta, phi) has ellipsoid coordinates
    r (sin theta cos(phi + dphi), sin theta sin(phi + dphi), cos theta).

    A cell whose centre value g = sqrt((x/a)^2 + (y/b)^2 + (z/c)^2) differs
    from 1 by more than (cell extent) / min(a, b, c) lies wholly inside or
    outside (g changes by at most |dx| / min(a, b, c)); it takes the centre's
    value.  The other cells average the indicator over a q x q x q product
    rule uniform in volume (r^3, cos theta, phi)."""
    a, b, c = (float(v) for v in axes)
    amin = min(a, b, c)
    cd, sd = math.cos(dphi), math.sin(dphi)
    th_e, ph_e = angular_cell_edges(spec)
    dth, dph = th_e[1] - th_e[0], ph_e[1] - ph_e[0]
    rm, rp = spec.r_edges[:-1], spec.r_edges[1:]
    extent = (rp - rm) + rp * (dth + dph)                      # bounds twice the half-diagonal
    r_c, units = cell_centres(spec)

    def g_of(x, y, z):
        xe, ye = cd * x - sd * y, sd * x + cd * y
        return np.sqrt((xe / a) ** 2 + (ye / b) ** 2 + (z / c) ** 2)

    gq, gw = np.polynomial.legendre.leggauss(q)
    u, uw = 0.5 * (gq + 1.0), 0.5 * gw
    out = {"yang": None}
    for patch in patches(spec):
        v = units[patch]
        gc = g_of(*(r_c[:, None, None] * v[k][None] for k in range(3)))
        rho = np.where(gc <= 1.0, rho0, 0.0)
        cut = np.abs(gc - 1.0) <= extent[:, None, None] / amin
        i_idx, j_idx, k_idx = np.nonzero(cut)
        if i_idx.size:
            r3m, r3p = rm[i_idx] ** 3, rp[i_idx] ** 3
            cm, cp = np.cos(th_e[j_idx]), np.cos(th_e[j_idx + 1])
            acc = np.zeros(i_idx.size)
            for ia in range(q):
                rr = np.cbrt(r3m + (r3p - r3m) * u[ia])
                for ib in range(q):
                    ct = cm + (cp - cm) * u[ib]
                    st = np.sqrt(np.clip(1.0 - ct * ct, 0.0, None))
                    for ic in range(q):
                        ph = ph_e[k_idx] + dph * u[ic]
                        x, y, z = st * np.cos(ph), st * np.sin(ph), ct
                        if patch == "yang":
                            x, y, z = -x, z, y
                        ind = g_of(rr * x, rr * y, rr * z) <= 1.0
                        acc += uw[ia] * uw[ib] * uw[ic] * ind
            rho[i_idx, j_idx, k_idx] = rho0 * acc
        out[patch] = rho
    return out["yin"], out["yang"]


def density_for(spec: GridSpec, seed: int | None = None):
    """Default density of a named grid."""
    if spec.name == "tiny":
        return tiny_density(spec)
    if spec.name == "mid":
        return oblate_density(spec, 1 if seed is None else seed)
    return pns_density(spec, 2 if seed is None else seed)


# ---------------------------------------------------------------------------
# batched workload: many fields of uneven size
# ---------------------------------------------------------------------------

_ANGULAR = [(45, 135), (60, 180), (90, 270)]


def batched_specs(n_fields: int = 64, first_seed: int = 100):
    """Fields of uneven size: n_r ~ U{100..600}, 2 / 1.5 / 1 degree cells,
    l_max ~ U{10..40}, eps scale ~ U(0.01, 0.1); field f uses seed first_seed + f."""
    out = []
    for f in range(n_fields):
        rng = np.random.default_rng(first_seed + f)
        n_r = int(rng.integers(100, 601))
        n_t, n_p = _ANGULAR[int(rng.integers(0, 3))]
        lmax = int(rng.integers(10, 41))
        eps_scale = float(rng.uniform(0.01, 0.1))
        spec = GridSpec(f"field{f}", np.logspace(-4, 0, n_r + 1), n_t, n_p, 0.0, 0.0, lmax)
        out.append((spec, first_seed + f, eps_scale))
    return out
