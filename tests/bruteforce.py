"""Brute-force O(N^2) evaluation of the discrete Yin-Yang potential (test helper).

Independent of the oracle's tables: it never uses P_l^m, T_j^(lm), C/S, the
radial closed forms or the angle transform.  For every target point and
every weighted source cell it sums

    Phi(x) = -G sum_cells rho w sum_{l <= lmax} int_shell r'^2 (r_<^l / r_>^(l+1)) dr'
                                              * int_cell P_l(cos gamma) dOmega'

which is the same truncated expansion written through the Legendre addition
theorem (sum_m N^(lm) P_l^m P_l^m cos m(phi - phi') = P_l(cos gamma)).  The
radial integrals use Gauss-Legendre in r (smooth powers), the angular ones a
q x q Gauss-Legendre rule per cell in (theta, phi); sources of the Yang patch
are placed in the global (Yin) frame by the Cartesian map (x,y,z)->(-x,z,y).
Passing ``lmax=None`` sums the exact Green's function 1/|x - x'| instead,
with a radial Gauss rule (then only a convergence check).
"""

from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg


def _patches(spec):
    return ("yin",) if getattr(spec, "polar", False) else ("yin", "yang")


def _edges(spec):
    if getattr(spec, "polar", False):       # one patch over the sphere, global frame
        return (math.pi / spec.n_theta * np.arange(spec.n_theta + 1),
                2 * math.pi / spec.n_phi * np.arange(spec.n_phi + 1))
    dth = (math.pi / 2 + 2 * spec.delta_theta) / spec.n_theta
    dph = (3 * math.pi / 2 + 2 * spec.delta_phi) / spec.n_phi
    te = math.pi / 4 - spec.delta_theta + dth * np.arange(spec.n_theta + 1)
    pe = -3 * math.pi / 4 - spec.delta_phi + dph * np.arange(spec.n_phi + 1)
    return te, pe


def _to_global(v, patch):
    return v if patch == "yin" else np.stack([-v[0], v[2], v[1]])


def source_points(spec, q=16):
    """Unit vectors [3, n_cells, q*q] (global frame) and weights [n_cells, q*q]
    (dOmega quadrature weights) of the cells of each patch."""
    te, pe = _edges(spec)
    g, gw = npleg.leggauss(q)
    out = {}
    for patch in _patches(spec):
        th = 0.5 * (te[:-1, None] + te[1:, None]) + 0.5 * (te[1:, None] - te[:-1, None]) * g[None]
        ph = 0.5 * (pe[:-1, None] + pe[1:, None]) + 0.5 * (pe[1:, None] - pe[:-1, None]) * g[None]
        wt = 0.5 * (te[1:, None] - te[:-1, None]) * gw[None] * np.sin(th)       # [n_t, q]
        wp = 0.5 * (pe[1:, None] - pe[:-1, None]) * gw[None]                     # [n_p, q]
        T = th[:, None, :, None]
        P = ph[None, :, None, :]
        x = np.sin(T) * np.cos(P)
        y = np.sin(T) * np.sin(P)
        z = np.cos(T) * np.ones_like(P)
        v = np.stack([np.broadcast_to(x, (spec.n_theta, spec.n_phi, q, q)),
                      np.broadcast_to(y, (spec.n_theta, spec.n_phi, q, q)),
                      np.broadcast_to(z, (spec.n_theta, spec.n_phi, q, q))])
        v = _to_global(v.reshape(3, spec.n_theta * spec.n_phi, q * q), patch)
        W = (wt[:, None, :, None] * wp[None, :, None, :]).reshape(spec.n_theta * spec.n_phi, q * q)
        out[patch] = (v, W)
    return out


def target_frame(spec, patch, j, k):
    """Global-frame unit vectors e_r, e_theta, e_phi at the centre of cell (j, k)."""
    te, pe = _edges(spec)
    th = 0.5 * (te[j] + te[j + 1])
    ph = 0.5 * (pe[k] + pe[k + 1])
    e_r = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    e_t = np.array([math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), -math.sin(th)])
    e_p = np.array([-math.sin(ph), math.cos(ph), 0.0])
    return [_to_global(e, patch) for e in (e_r, e_t, e_p)]


def _radial_factors(r_edges, r, lmax, qr=24):
    """int_shell r'^2 r_<^l / r_>^(l+1) dr' and its derivative in r, for each
    shell i and l (shells entirely inside or outside r, since r is an edge)."""
    g, gw = npleg.leggauss(qr)
    rm, rp = r_edges[:-1], r_edges[1:]
    rs = 0.5 * (rm + rp)[:, None] + 0.5 * (rp - rm)[:, None] * g[None]
    ws = 0.5 * (rp - rm)[:, None] * gw[None]
    inner = (rp <= r * (1 + 1e-14))[:, None]
    F = np.zeros((lmax + 1, rm.size))
    dF = np.zeros((lmax + 1, rm.size))
    for l in range(lmax + 1):
        val = np.where(inner, rs ** (l + 2) / r ** (l + 1), r ** l * rs ** (1 - l))
        der = np.where(inner, -(l + 1) * rs ** (l + 2) / r ** (l + 2),
                       (l * r ** (l - 1) if l > 0 else 0.0) * rs ** (1 - l))
        F[l] = (val * ws).sum(axis=1)
        dF[l] = (der * ws).sum(axis=1)
    return F, dF


def potential_and_gradient(spec, w, rho, targets, q=16):
    """Phi and -grad Phi (target-local spherical components) at targets.

    rho: {"yin": [n_r, n_t, n_p], "yang": ...}; w: [n_t, n_p] weights;
    targets: list of (patch, n, j, k), n = 0..n_r-1 meaning r = r_edges[n+1].
    Returns (phi [T], grad [T, 3]).
    """
    L = spec.lmax
    src = source_points(spec, q)
    wflat = w.reshape(-1)
    phis, grads = [], []
    for patch_t, n, j, k in targets:
        r = spec.r_edges[n + 1]
        e_r, e_t, e_p = target_frame(spec, patch_t, j, k)
        F, dF = _radial_factors(spec.r_edges, r, L)
        phi = 0.0
        grad = np.zeros(3)
        for patch_s in _patches(spec):
            v, W = src[patch_s]
            cg = np.einsum("c,cnq->nq", e_r, v)
            I = np.empty((L + 1, cg.shape[0]))
            J = np.empty((L + 1, 3, cg.shape[0]))
            for l in range(L + 1):
                c = np.zeros(l + 1)
                c[l] = 1.0
                Pl = npleg.legval(cg, c)
                dPl = npleg.legval(cg, npleg.legder(c)) if l > 0 else np.zeros_like(cg)
                I[l] = (Pl * W).sum(axis=1)
                tang = v - cg[None] * e_r[:, None, None]
                J[l] = np.einsum("nq,cnq->cn", dPl * W, tang)
            rw = rho[patch_s].reshape(spec.n_r, -1) * wflat[None]      # [i, cell]
            S_I = rw @ I.T                                             # [i, l]
            S_J = np.einsum("ic,lxc->ilx", rw, J)                      # [i, l, 3]
            phi += -spec.G * np.einsum("li,il->", F, S_I)
            dphi_dr = -spec.G * np.einsum("li,il->", dF, S_I)
            grad_tan = -spec.G * np.einsum("li,ilx->x", F, S_J) / r
            gvec = dphi_dr * e_r + grad_tan
            grad += gvec
        phis.append(phi)
        grads.append([-grad @ e_r, -grad @ e_t, -grad @ e_p])
    return np.array(phis), np.array(grads)


def green_potential(spec, w, rho, targets, q=8, qr=8):
    """Phi from the exact kernel 1/|x - x'| (no truncation), midpoint-free
    Gauss rule per cell in (r, theta, phi); for convergence checks only."""
    src = source_points(spec, q)
    g, gw = npleg.leggauss(qr)
    rm, rp = spec.r_edges[:-1], spec.r_edges[1:]
    rs = 0.5 * (rm + rp)[:, None] + 0.5 * (rp - rm)[:, None] * g[None]
    ws = 0.5 * (rp - rm)[:, None] * gw[None] * rs ** 2
    out = []
    for patch_t, n, j, k in targets:
        r = spec.r_edges[n + 1]
        e_r = target_frame(spec, patch_t, j, k)[0]
        x = r * e_r
        phi = 0.0
        for patch_s in _patches(spec):
            v, W = src[patch_s]
            wcell = W * w.reshape(-1)[:, None]                          # [cell, q2]
            for i in range(spec.n_r):
                pts = rs[i][None, None, :, None] * v[:, :, None, :]      # [3, cell, qr, q2]
                d = np.sqrt(((pts - x[:, None, None, None]) ** 2).sum(axis=0))
                kern = (ws[i][None, :, None] * wcell[:, None, :] / d).sum(axis=(1, 2))
                phi += -spec.G * (rho[patch_s][i].reshape(-1) * kern).sum()
        out.append(phi)
    return np.array(out)
