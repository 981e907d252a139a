"""Plain float64 restatement of the Yin-Yang multipole gravity solver.

TEST INFRASTRUCTURE: the independent CPU oracle the CUDA library is checked
against.  Only tests/, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference arm may import it.  It shares no code with the
library.

Method: Almanstötter, Melson, Janka & Müller (2018), arXiv:1806.04593, which
applies the multipole solver of Müller & Steinmetz (1995) to the two patches
of the Yin-Yang grid.  The steps below follow the paper's order and notation:

* §2 (Eqs. potential, phiin_tot, phiout_tot, rin, rout, tlm and the closed
  forms for C_k^(m), S_k^(m)): the cell integrals of the discretised problem.
* Appendix: the recurrences for T_j^(lm), evaluated in the order printed.
* §3 (Eqs. phiin, phiout, ac, as): separation into the angular sums A_C, A_S
  and the radial inner / outer sums.
* §4: patch geometry, the Yin -> Yang angle map (Eqs. trafotheta, trafophi),
  the overlap surface weights w_jk and their 2*pi identity, the weighted
  per-patch sums and the sum of the four potentials.

Library primitives used as steps: numpy matmul / cumsum for the plain sums
the equations write out, scipy.integrate.quad (adaptive Gauss-Kronrod) for
the cut-cell areas.  Nothing is blocked, fused or reordered beyond that.

Readings where the paper is silent, ambiguous or garbled:

R1  T^(22) seed (Appendix): the printed seed is missing a bracket.  We use
    1/4 [(cos 3t+ - cos 3t-) - 9 (cos t+ - cos t-)], which is the exact
    integral of sin(t) P_2^2(cos t) and equals the T^(ll) recurrence at l=2.
R2  phi_Yang (Eq. trafophi): the bare arctan is taken quadrant-correct,
    atan2(cos t, -sin t cos p); theta_Yang = arccos(sin t sin p).
R3  Evaluation points (§2): radially the outer interface r_n^+ of zone n
    (n = 1..n_R, the paper evaluates at interfaces); angularly the cell-centre
    midpoints (theta_j, phi_k) of the target patch (the paper is silent).
R4  Overlap weights (§4): w_jk = 1 - f_jk / 2, f_jk the exact solid-angle
    fraction of cell jk inside the other patch's closed domain.  This gives
    1/2 inside the overlap, 1 outside, and sum(dOmega * w) = 2*pi per patch.
R5  Density is zero inside r_edges[0] (the innermost zone starts there).
R6  Associated Legendre functions carry the Condon-Shortley phase; this is
    the convention under which the paper's T^(11) seed is the integral of
    sin(t) P_1^1(cos t).
R7  -grad(Phi) is returned in the target patch's local spherical basis
    (g_r, g_theta, g_phi); the paper computes Phi only.  The radial derivative
    at r_n^+ is d/dr[r^-(l+1) C(r) + r^l D(r)] = (-(l+1) c_n + l d_n) / r_n
    (the density terms cancel), the angular ones differentiate the series.
R8  T_j^(lm) (Eq. tlm) has a plain definition, an integral; the oracle
    evaluates that definition by a converged Gauss-Legendre rule.  The
    Appendix recurrences are kept as :func:`polar_integrals_appendix` and
    agree with it to rounding, except that the T^(ll) diagonal amplifies
    rounding by ~(1/sin^2 theta)^(l/2) (6e-12 relative at l = 25 on 1-degree
    cells, 1e-6 at l = 40 on 7.5-degree cells).
R10 Full spherical polar grid (§2): the paper does not state the cell
    layout; we take uniform cells, theta_j^+- = (j, j+1) pi / n_theta and
    phi_k^+- = (k, k+1) 2 pi / n_phi, one patch with w = 1, evaluated at its
    own cell centres (R3).
"""

from __future__ import annotations

import math
import warnings

import numpy as np
from scipy import integrate


# ---------------------------------------------------------------------------
# §4 patch geometry and the Yin <-> Yang map
# ---------------------------------------------------------------------------

def angular_edges(n_theta, n_phi, delta_theta, delta_phi):
    """Cell edges of one patch in its own local angles (§4 patch intervals).

    theta spans [pi/4 - d_theta, 3pi/4 + d_theta] in n_theta equal cells and
    phi spans [-3pi/4 - d_phi, 3pi/4 + d_phi] in n_phi equal cells.
    """
    th0 = math.pi / 4 - delta_theta
    th1 = 3 * math.pi / 4 + delta_theta
    ph0 = -3 * math.pi / 4 - delta_phi
    ph1 = 3 * math.pi / 4 + delta_phi
    theta_edges = th0 + (th1 - th0) / n_theta * np.arange(n_theta + 1)
    phi_edges = ph0 + (ph1 - ph0) / n_phi * np.arange(n_phi + 1)
    return theta_edges, phi_edges


def other_patch_angles(theta, phi):
    """Angles of a point in the other patch's frame (Eqs. trafotheta, trafophi).

    The same formulas map Yin -> Yang and Yang -> Yin (reading R2 for phi).
    """
    st, ct = np.sin(theta), np.cos(theta)
    sp, cp = np.sin(phi), np.cos(phi)
    theta_o = np.arccos(np.clip(st * sp, -1.0, 1.0))
    phi_o = np.arctan2(ct, -st * cp)
    return theta_o, phi_o


def other_patch_cartesian(v):
    """Cartesian components in the other patch's frame: (x, y, z) -> (-x, z, y).

    This linear map reproduces Eqs. trafotheta / trafophi (cos theta' = y/r,
    tan phi' = z / (-x)); it is its own inverse and has determinant +1.
    """
    v = np.asarray(v)
    return np.stack([-v[0], v[2], v[1]])


def spherical_basis(theta, phi):
    """Unit vectors e_r, e_theta, e_phi (Cartesian components, local frame)."""
    st, ct = np.sin(theta), np.cos(theta)
    sp, cp = np.sin(phi), np.cos(phi)
    e_r = np.stack([st * cp, st * sp, ct])
    e_t = np.stack([ct * cp, ct * sp, -st])
    e_p = np.stack([-sp, cp, np.zeros_like(st)])
    return e_r, e_t, e_p


# ---------------------------------------------------------------------------
# §4 overlap surface weights (reading R4)
# ---------------------------------------------------------------------------

def _other_patch_theta_measure(phi, th_lo, th_hi, c1, t2):
    """Integral of sin(theta) over theta in [th_lo, th_hi] restricted to the
    other patch's domain, at fixed azimuth phi (own-patch angles).

    In own-patch Cartesian coordinates the other patch's domain is
    |y| <= c1 r with c1 = cos(pi/4 - d_theta)          (theta' limits)
    and not (x > 0 and |z| < t2 x) with t2 = tan(pi/4 - d_phi)  (phi' limits),
    which follows from cos theta' = y/r and phi' = atan2(z, -x).
    """
    s = abs(math.sin(phi))
    if s <= c1:
        allowed = [(0.0, math.pi)]
    else:
        a = math.asin(c1 / s)
        allowed = [(0.0, a), (math.pi - a, math.pi)]
    cphi = math.cos(phi)
    pieces = []
    if cphi > 0.0:
        b = math.atan2(1.0, t2 * cphi)       # |cot theta| < t2 cos phi  <=>  b < theta < pi - b
        for lo, hi in allowed:
            if min(hi, b) > lo:
                pieces.append((lo, min(hi, b)))
            if hi > max(lo, math.pi - b):
                pieces.append((max(lo, math.pi - b), hi))
    else:
        pieces = allowed
    total = 0.0
    for lo, hi in pieces:
        lo = max(lo, th_lo)
        hi = min(hi, th_hi)
        if hi > lo:
            total += math.cos(lo) - math.cos(hi)
    return total


def _weight_breakpoints(ph_lo, ph_hi, th_lo, th_hi, c1, t2):
    """Azimuths in (ph_lo, ph_hi) where the integrand above has a kink or a
    square-root endpoint: a domain boundary meets a theta edge, the boundaries
    meet each other, |sin phi| = c1, or cos phi = 0."""
    cands = []

    def at_abs_sin(v):
        if 0.0 <= v <= 1.0:
            a = math.asin(v)
            cands.extend([a, -a, math.pi - a, a - math.pi])

    def at_cos(v):
        if -1.0 <= v <= 1.0:
            a = math.acos(v)
            cands.extend([a, -a])

    at_abs_sin(c1)
    at_cos(0.0)
    for te in (th_lo, th_hi):
        st = math.sin(te)
        if st > 0.0:
            at_abs_sin(c1 / st)
            cot = math.cos(te) / st
            at_cos(cot / t2)
            at_cos(-cot / t2)
    at_cos(math.sqrt((1.0 - c1 * c1) / (1.0 + c1 * c1 * t2 * t2)))
    return sorted({p for p in cands if ph_lo < p < ph_hi})


def overlap_weights(theta_edges, phi_edges, delta_theta, delta_phi):
    """Surface weights w_jk of one patch (§4), reading R4.

    w_jk = 1 - f_jk / 2 where f_jk is the fraction of the cell's solid angle
    dOmega_jk = (cos theta_j^- - cos theta_j^+)(phi_k^+ - phi_k^-) that lies in
    the other patch.  The cut area is integral dphi of the theta measure above,
    done by adaptive Gauss-Kronrod with the kinks as breakpoints.  The weights
    are the same on both patches (identical local coordinates).
    """
    c1 = math.cos(math.pi / 4 - delta_theta)
    t2 = math.tan(math.pi / 4 - delta_phi)
    n_t, n_p = len(theta_edges) - 1, len(phi_edges) - 1
    w = np.empty((n_t, n_p))
    for j in range(n_t):
        th_lo, th_hi = float(theta_edges[j]), float(theta_edges[j + 1])
        band = math.cos(th_lo) - math.cos(th_hi)
        for k in range(n_p):
            ph_lo, ph_hi = float(phi_edges[k]), float(phi_edges[k + 1])
            cell = band * (ph_hi - ph_lo)
            pts = _weight_breakpoints(ph_lo, ph_hi, th_lo, th_hi, c1, t2)
            with warnings.catch_warnings():
                warnings.simplefilter("ignore", integrate.IntegrationWarning)
                area, err = integrate.quad(
                    _other_patch_theta_measure, ph_lo, ph_hi,
                    args=(th_lo, th_hi, c1, t2), points=pts or None,
                    epsabs=1e-15 * cell, epsrel=1e-14, limit=400)
            if err > 1e-12 * cell:
                raise RuntimeError(f"cut-cell area of ({j},{k}) not converged: {err}")
            w[j, k] = 1.0 - 0.5 * (area / cell)
    return w


# ---------------------------------------------------------------------------
# §2 / Appendix: Legendre functions and the cell integrals
# ---------------------------------------------------------------------------

def assoc_legendre(lmax, x, s):
    """P_l^m(x) for 0 <= m <= l <= lmax with the Condon-Shortley phase (R6).

    x = cos(theta), s = sin(theta) >= 0 (passed separately so that the seed
    (1 - x^2)^(m/2) = s^m keeps full precision near the poles).  Standard
    recurrences: P_m^m = -(2m-1) s P_{m-1}^{m-1}, P_{m+1}^m = (2m+1) x P_m^m,
    (l - m) P_l^m = (2l - 1) x P_{l-1}^m - (l + m - 1) P_{l-2}^m.
    Returns shape (lmax+1, lmax+1) + x.shape; entries with m > l are zero.
    """
    x = np.asarray(x, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    P = np.zeros((lmax + 1, lmax + 1) + x.shape)
    P[0, 0] = 1.0
    for m in range(1, lmax + 1):
        P[m, m] = -(2 * m - 1) * s * P[m - 1, m - 1]
    for m in range(lmax):
        P[m + 1, m] = (2 * m + 1) * x * P[m, m]
    for m in range(lmax + 1):
        for l in range(m + 2, lmax + 1):
            P[l, m] = ((2 * l - 1) * x * P[l - 1, m] - (l + m - 1) * P[l - 2, m]) / (l - m)
    return P


def dlegendre_dtheta(P):
    """d/dtheta P_l^m(cos theta), pole-safe (no division by sin theta).

    Condon-Shortley identities: dP_l^0/dtheta = P_l^1 and, for m >= 1,
    dP_l^m/dtheta = (P_l^(m+1) - (l + m)(l - m + 1) P_l^(m-1)) / 2.
    ``P`` is the array from :func:`assoc_legendre`.
    """
    lmax = P.shape[0] - 1
    dP = np.zeros_like(P)
    for l in range(1, lmax + 1):
        dP[l, 0] = P[l, 1]
        for m in range(1, l + 1):
            up = P[l, m + 1] if m + 1 <= l else 0.0
            dP[l, m] = 0.5 * (up - (l + m) * (l - m + 1) * P[l, m - 1])
    return dP


def legendre_m_over_sin(P):
    """m P_l^m(cos theta) / sin theta, pole-safe.

    Condon-Shortley identity, m >= 1:
    m P_l^m / sin theta = -(P_{l-1}^(m+1) + (l + m - 1)(l + m) P_{l-1}^(m-1)) / 2;
    zero for m = 0.
    """
    lmax = P.shape[0] - 1
    Q = np.zeros_like(P)
    for l in range(1, lmax + 1):
        for m in range(1, l + 1):
            up = P[l - 1, m + 1] if m + 1 <= l - 1 else 0.0
            Q[l, m] = -0.5 * (up + (l + m - 1) * (l + m) * P[l - 1, m - 1])
    return Q


def normalisation(lmax):
    """N^(lm) = (l - m)!/(l + m)! * 2/delta^(m), delta^(0) = 2, else 1 (§2)."""
    N = np.zeros((lmax + 1, lmax + 1))
    for l in range(lmax + 1):
        for m in range(l + 1):
            N[l, m] = (math.factorial(l - m) / math.factorial(l + m)) * (1.0 if m == 0 else 2.0)
    return N


def polar_integrals(lmax, theta_edges):
    """T_j^(lm) = int_{theta_j^-}^{theta_j^+} sin(t) P_l^m(cos t) dt (Eq. tlm),
    written out as its definition (reading R8).

    sin(t) P_l^m(cos t) is a trigonometric polynomial of degree l + 1 in t, so
    a Gauss-Legendre rule with lmax + 32 nodes per cell integrates it to
    rounding.  Returns shape (lmax+1, lmax+1, n_theta); zero for m > l.
    """
    te = np.asarray(theta_edges, dtype=np.float64)
    nodes, weights = np.polynomial.legendre.leggauss(lmax + 32)
    T = np.zeros((lmax + 1, lmax + 1, te.size - 1))
    for j in range(te.size - 1):
        half = 0.5 * (te[j + 1] - te[j])
        t = 0.5 * (te[j] + te[j + 1]) + half * nodes
        P = assoc_legendre(lmax, np.cos(t), np.sin(t))
        T[:, :, j] = P @ (half * weights * np.sin(t))
    return T


def polar_integrals_appendix(lmax, theta_edges):
    """T_j^(lm) by the Appendix recurrences in the printed order (T^(22) per
    reading R1).  Exact in exact arithmetic; in floating point the T^(ll)
    recurrence multiplies the rounding error of T^(l-2,l-2) by about
    1 / sin^2(theta) per step, so the diagonal loses digits at large l
    (reading R8).  Kept as the paper's route and checked against
    :func:`polar_integrals`.
    """
    tm = np.asarray(theta_edges[:-1], dtype=np.float64)   # theta_j^-
    tp = np.asarray(theta_edges[1:], dtype=np.float64)    # theta_j^+
    xm, xp = np.cos(tm), np.cos(tp)
    sm, sp = np.sin(tm), np.sin(tp)
    Pm = assoc_legendre(lmax + 1, xm, sm)
    Pp = assoc_legendre(lmax + 1, xp, sp)
    T = np.zeros((lmax + 1, lmax + 1, tm.size))
    # T^(00)
    T[0, 0] = Pm[1, 0] - Pp[1, 0]
    # T^(l0), l > 0
    for l in range(1, lmax + 1):
        T[l, 0] = (Pp[l - 1, 0] - Pm[l - 1, 0] + Pm[l + 1, 0] - Pp[l + 1, 0]) / (2 * l + 1)
    # T^(11)
    if lmax >= 1:
        T[1, 1] = 0.5 * (tm - tp + 0.5 * (np.sin(2 * tp) - np.sin(2 * tm)))
    # T^(22), reading R1
    if lmax >= 2:
        T[2, 2] = 0.25 * ((np.cos(3 * tp) - np.cos(3 * tm)) - 9.0 * (np.cos(tp) - np.cos(tm)))
    # T^(ll), l >= 3, from T^(l-2, l-2)
    for l in range(3, lmax + 1):
        T[l, l] = (xm * Pm[l, l] - xp * Pp[l, l]
                   + l * (2 * l - 3) * (2 * l - 1) * T[l - 2, l - 2]) / (l + 1)
    # T^(l, l-1), l >= 2 (l = 1 is the m = 0 column above)
    for l in range(2, lmax + 1):
        T[l, l - 1] = -(sp * Pp[l, l] - sm * Pm[l, l]) / (l + 1)
    # T^(lm), m >= 1, l >= m + 2, from T^(l-2, m)
    for m in range(1, lmax + 1):
        for l in range(m + 2, lmax + 1):
            T[l, m] = ((2 * l - 1) * (sp * sp * Pp[l - 1, m] - sm * sm * Pm[l - 1, m])
                       + (l - 2) * (l + m - 1) * T[l - 2, m]) / ((l + 1) * (l - m))
    return T


def azimuthal_integrals(lmax, phi_edges):
    """C_k^(m) = int cos(m phi) dphi and S_k^(m) = int sin(m phi) dphi over
    cell k, in the closed forms of §2.  Shapes (lmax+1, n_phi)."""
    pm = np.asarray(phi_edges[:-1], dtype=np.float64)
    pp = np.asarray(phi_edges[1:], dtype=np.float64)
    C = np.zeros((lmax + 1, pm.size))
    S = np.zeros((lmax + 1, pm.size))
    C[0] = pp - pm
    for m in range(1, lmax + 1):
        C[m] = (np.sin(m * pp) - np.sin(m * pm)) / m
        S[m] = (np.cos(m * pm) - np.cos(m * pp)) / m
    return C, S


def radial_integrals(lmax, r_edges):
    """R_in,i^(l) and R_out,i^(l) of Eqs. rin / rout, shapes (lmax+1, n_R).

    R_out of a zone starting at r = 0 diverges for l >= 2; it never enters a
    sum (outer sums start at i = n + 1 >= 2) and is stored as NaN.
    """
    r = np.asarray(r_edges, dtype=np.float64)
    rm, rp = r[:-1], r[1:]
    Rin = np.zeros((lmax + 1, rm.size))
    Rout = np.zeros((lmax + 1, rm.size))
    with np.errstate(divide="ignore", invalid="ignore"):
        for l in range(lmax + 1):
            Rin[l] = (rp ** (l + 3) - rm ** (l + 3)) / (l + 3)
            if l == 2:
                Rout[l] = np.log(rp) - np.log(rm)
            else:
                Rout[l] = (rp ** (2 - l) - rm ** (2 - l)) / (2 - l)
    Rout[2:, rm == 0.0] = np.nan
    return Rin, Rout


# ---------------------------------------------------------------------------
# The solver
# ---------------------------------------------------------------------------

class OracleGrid:
    """Constant terms of one Yin-Yang grid (§3, last paragraph) plus the solve.

    Arrays are indexed [i or n][j][k] (radial, theta, phi) per patch; moment
    arrays are [i][l][m] with separate cos (C) and sin (S) parts.
    """

    def __init__(self, r_edges, n_theta, n_phi, delta_theta, delta_phi, lmax, G=1.0):
        self.r_edges = np.asarray(r_edges, dtype=np.float64)
        self.n_r = self.r_edges.size - 1
        self.n_theta, self.n_phi = int(n_theta), int(n_phi)
        self.delta_theta, self.delta_phi = float(delta_theta), float(delta_phi)
        self.lmax = int(lmax)
        self.G = float(G)
        self.theta_edges, self.phi_edges = angular_edges(n_theta, n_phi, delta_theta, delta_phi)
        self._constant_terms(overlap_weights(self.theta_edges, self.phi_edges, delta_theta, delta_phi))

    def _constant_terms(self, w):
        """The density-independent factors of Eqs. ac/as, rin/rout and
        potential for the cell edges set on self, with surface weights w."""
        n_theta, n_phi = self.n_theta, self.n_phi
        self.theta_c = 0.5 * (self.theta_edges[:-1] + self.theta_edges[1:])
        self.phi_c = 0.5 * (self.phi_edges[:-1] + self.phi_edges[1:])
        L = self.lmax
        self.w = w
        self.T = polar_integrals(L, self.theta_edges)
        self.C, self.S = azimuthal_integrals(L, self.phi_edges)
        self.R_in, self.R_out = radial_integrals(L, self.r_edges)
        self.N = normalisation(L)
        # Density-independent factor of Eqs. ac/as with the weight of §4:
        # (w_jk T_j^(lm) C_k^(m)) and (w_jk T_j^(lm) S_k^(m)), rows (j,k), cols (l,m).
        WT = self.w[:, :, None, None] * np.transpose(self.T, (2, 0, 1))[:, None, :, :]
        self.B_C = (WT * np.transpose(self.C)[None, :, None, :]).reshape(n_theta * n_phi, -1)
        self.B_S = (WT * np.transpose(self.S)[None, :, None, :]).reshape(n_theta * n_phi, -1)
        # target cell centres, own frame (R3)
        tt, pp = np.meshgrid(self.theta_c, self.phi_c, indexing="ij")
        self.target_theta = tt.reshape(-1)
        self.target_phi = pp.reshape(-1)

    # -- §3 / §4 analysis ----------------------------------------------------
    def analysis(self, rho):
        """A_C,i^(lm) and A_S,i^(lm) of one patch (§4 weighted Eqs. ac/as)."""
        rho = np.asarray(rho, dtype=np.float64).reshape(self.n_r, -1)
        L1 = self.lmax + 1
        A_C = (rho @ self.B_C).reshape(self.n_r, L1, L1)
        A_S = (rho @ self.B_S).reshape(self.n_r, L1, L1)
        return A_C, A_S

    # -- §3 radial sums (Eqs. phiin / phiout at r = r_n^+) ---------------------
    def radial_sums(self, A_C, A_S):
        """Coefficients of cos(m phi) and sin(m phi) in Phi_in + Phi_out at the
        interfaces r_n^+ (n = 1..n_R), and of their radial derivative (R7).

        Phi_in = r^-(l+1) sum_{i<=n} R_in,i (...), Phi_out = r^l sum_{i>n} R_out,i (...).
        """
        L = self.lmax
        r = self.r_edges[1:]
        l = np.arange(L + 1, dtype=np.float64)
        out = {}
        for name, A in (("C", A_C), ("S", A_S)):
            t_in = self.R_in.T[:, :, None] * A                       # [i, l, m]
            inner = np.cumsum(t_in, axis=0)                           # sum_{i <= n}
            with np.errstate(invalid="ignore"):
                t_out = self.R_out.T[:, :, None] * A
            t_out[0] = 0.0                       # shell 1 is never in an outer sum (i > n >= 1)
            outer = np.zeros_like(t_out)
            outer[:-1] = np.cumsum(t_out[::-1], axis=0)[::-1][1:]     # sum_{i > n}
            c = r[:, None, None] ** (-(l[None, :, None] + 1)) * inner
            d = r[:, None, None] ** (l[None, :, None]) * outer
            out["U_" + name] = c + d
            out["dU_" + name] = (-(l[None, :, None] + 1) * c + l[None, :, None] * d) / r[:, None, None]
        return out

    # -- §2 Eq. potential evaluated at given angles ---------------------------
    def _basis(self, theta, phi):
        L = self.lmax
        P = assoc_legendre(L, np.cos(theta), np.sin(theta))
        m = np.arange(L + 1)
        cosm = np.cos(m[:, None] * phi[None, :])
        sinm = np.sin(m[:, None] * phi[None, :])
        return P, cosm, sinm

    def evaluate(self, coef, theta, phi):
        """-G sum_lm N^(lm) P_l^m(cos theta)[cos(m phi) U_C + sin(m phi) U_S] at
        every interface radius (rows) and every given angle (columns)."""
        theta = np.atleast_1d(np.asarray(theta, dtype=np.float64))
        phi = np.atleast_1d(np.asarray(phi, dtype=np.float64))
        P, cosm, sinm = self._basis(theta, phi)
        NP = self.N[:, :, None] * P
        bC = (NP * cosm[None, :, :]).reshape(-1, theta.size)
        bS = (NP * sinm[None, :, :]).reshape(-1, theta.size)
        UC = coef["U_C"].reshape(self.n_r, -1)
        US = coef["U_S"].reshape(self.n_r, -1)
        return -self.G * (UC @ bC + US @ bS)

    def evaluate_gradient(self, coef, theta, phi):
        """-grad(Phi) of one source patch at given own-frame angles, as
        Cartesian components in that frame: shape (3, n_R, n_points).

        d/dr uses the dU coefficients (R7); (1/r) d/dtheta differentiates
        P_l^m; (1/(r sin theta)) d/dphi differentiates cos / sin(m phi).
        """
        theta = np.atleast_1d(np.asarray(theta, dtype=np.float64))
        phi = np.atleast_1d(np.asarray(phi, dtype=np.float64))
        P, cosm, sinm = self._basis(theta, phi)
        NP = self.N[:, :, None] * P
        NdP = self.N[:, :, None] * dlegendre_dtheta(P)
        NmPs = self.N[:, :, None] * legendre_m_over_sin(P)
        flat = lambda a: a.reshape(-1, theta.size)
        UC, US = coef["U_C"].reshape(self.n_r, -1), coef["U_S"].reshape(self.n_r, -1)
        dUC, dUS = coef["dU_C"].reshape(self.n_r, -1), coef["dU_S"].reshape(self.n_r, -1)
        d_r = -self.G * (dUC @ flat(NP * cosm[None]) + dUS @ flat(NP * sinm[None]))
        d_t = -self.G * (UC @ flat(NdP * cosm[None]) + US @ flat(NdP * sinm[None]))
        d_p_over_sin = -self.G * (UC @ flat(-NmPs * sinm[None]) + US @ flat(NmPs * cosm[None]))
        r = self.r_edges[1:][:, None]
        g_r, g_t, g_p = -d_r, -d_t / r, -d_p_over_sin / r
        e_r, e_t, e_p = spherical_basis(theta, phi)
        return (g_r[None] * e_r[:, None, :] + g_t[None] * e_t[:, None, :]
                + g_p[None] * e_p[:, None, :])

    # -- §4 the four potentials and their sums ---------------------------------
    def solve(self, rho_yin, rho_yang, gradient=False, cells=None):
        """Phi (and optionally -grad Phi) on both patches (§4).

        Phi(r_Yin) = Phi_Yin(r_Yin) + Phi_Yang(r_Yin), and likewise on Yang:
        the moments of each patch are evaluated at the target points expressed
        in that patch's angles.  ``cells`` optionally restricts the target
        angular cells (flat indices j*n_phi + k); all radii are returned.
        Returns dict with 'phi_yin', 'phi_yang' of shape (n_R, n_cells) (or
        (n_R, n_theta, n_phi) when cells is None) and 'grad_yin', 'grad_yang'
        of shape (3, ...) holding (g_r, g_theta, g_phi) (R7).
        """
        coef = {
            "yin": self.radial_sums(*self.analysis(rho_yin)),
            "yang": self.radial_sums(*self.analysis(rho_yang)),
        }
        th = self.target_theta if cells is None else self.target_theta[cells]
        ph = self.target_phi if cells is None else self.target_phi[cells]
        th_x, ph_x = other_patch_angles(th, ph)
        res = {}
        for q, p in (("yin", "yang"), ("yang", "yin")):
            phi = self.evaluate(coef[q], th, ph) + self.evaluate(coef[p], th_x, ph_x)
            res["phi_" + q] = phi
            if gradient:
                v_own = self.evaluate_gradient(coef[q], th, ph)
                v_other = other_patch_cartesian(self.evaluate_gradient(coef[p], th_x, ph_x))
                v = v_own + v_other
                e_r, e_t, e_p = spherical_basis(th, ph)
                res["grad_" + q] = np.stack([
                    np.einsum("cnp,cp->np", v, e_r),
                    np.einsum("cnp,cp->np", v, e_t),
                    np.einsum("cnp,cp->np", v, e_p),
                ])
        if cells is None:
            shp = (self.n_r, self.n_theta, self.n_phi)
            for key in list(res):
                res[key] = res[key].reshape(((3,) if key.startswith("grad") else ()) + shp)
        return res


class OraclePolarGrid(OracleGrid):
    """The full spherical polar grid of §2: one patch, theta_j^+- = (j, j+1)
    pi / n_theta and phi_k^+- = (k, k+1) 2 pi / n_phi, every cell counted once
    (w = 1), no second patch.  Eqs. potential, phiin_tot and phiout_tot with
    the sums over all cells of the sphere; the radial sums and the evaluation
    are those of :class:`OracleGrid`.
    """

    def __init__(self, r_edges, n_theta, n_phi, lmax, G=1.0):
        self.r_edges = np.asarray(r_edges, dtype=np.float64)
        self.n_r = self.r_edges.size - 1
        self.n_theta, self.n_phi = int(n_theta), int(n_phi)
        self.delta_theta = self.delta_phi = 0.0
        self.lmax = int(lmax)
        self.G = float(G)
        self.theta_edges = math.pi / self.n_theta * np.arange(self.n_theta + 1)
        self.phi_edges = 2.0 * math.pi / self.n_phi * np.arange(self.n_phi + 1)
        self._constant_terms(np.ones((self.n_theta, self.n_phi)))

    def solve(self, rho, gradient=False, cells=None):
        """Phi (and optionally -grad Phi in the local spherical basis, R7) at
        the interfaces r_n^+ and the cell centres (R3).  Returns 'phi' of
        shape (n_R, n_theta, n_phi) (or (n_R, n_cells) for a cell sample) and
        'grad' of shape (3, ...)."""
        coef = self.radial_sums(*self.analysis(rho))
        th = self.target_theta if cells is None else self.target_theta[cells]
        ph = self.target_phi if cells is None else self.target_phi[cells]
        res = {"phi": self.evaluate(coef, th, ph)}
        if gradient:
            v = self.evaluate_gradient(coef, th, ph)
            e_r, e_t, e_p = spherical_basis(th, ph)
            res["grad"] = np.stack([np.einsum("cnp,cp->np", v, e) for e in (e_r, e_t, e_p)])
        if cells is None:
            shp = (self.n_r, self.n_theta, self.n_phi)
            res["phi"] = res["phi"].reshape(shp)
            if gradient:
                res["grad"] = res["grad"].reshape((3,) + shp)
        return res

