"""Pins of the CPU oracle against values fixed by the paper and by mathematics.

None of these re-types an oracle formula: each compares the oracle with an
independent computation (quadrature, a library routine, a closed form, a
brute-force sum through the Legendre addition theorem) or with an identity the
paper states (the 2*pi weight sum of §4, the spherical test of §5).
"""

import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from scipy import special

import oracle
from oracle import yinyang
from paper_1806_04593_gb300 import inputs

from . import bruteforce as bf


def _gl(a, b, q):
    g, w = npleg.leggauss(q)
    return 0.5 * (a + b) + 0.5 * (b - a) * g, 0.5 * (b - a) * w


# ---------------------------------------------------------------------------
# Legendre functions
# ---------------------------------------------------------------------------

def test_assoc_legendre_matches_scipy_lpmv():
    rng = np.random.default_rng(3)
    th = rng.uniform(0.0, math.pi, 64)
    L = 40
    P = oracle.assoc_legendre(L, np.cos(th), np.sin(th))
    for l in range(L + 1):
        for m in range(l + 1):
            ref = special.lpmv(m, l, np.cos(th))
            scale = np.abs(ref).max() + 1e-300
            assert np.abs(P[l, m] - ref).max() <= 1e-12 * scale, (l, m)


def test_assoc_legendre_orthogonality():
    # int_{-1}^{1} P_l^m P_k^m dx = 2/(2l+1) (l+m)!/(l-m)! delta_lk; the product
    # is a polynomial of degree <= 2L, so the Gauss rule below is exact
    L = 30
    x, w = npleg.leggauss(L + 2)
    P = oracle.assoc_legendre(L, x, np.sqrt(1 - x * x))
    for m in range(L + 1):
        ls = np.arange(m, L + 1)
        Gm = np.einsum("q,aq,bq->ab", w, P[m:, m], P[m:, m])
        norm = np.array([2.0 / (2 * l + 1) * math.factorial(l + m) / math.factorial(l - m) for l in ls])
        scaled = Gm / np.sqrt(norm[:, None] * norm[None, :])
        assert np.abs(scaled - np.eye(ls.size)).max() <= 1e-12, m


def test_legendre_derivatives_against_finite_differences_and_division():
    L = 20
    rng = np.random.default_rng(4)
    th = rng.uniform(0.2, math.pi - 0.2, 40)
    h = 1e-5
    P = oracle.assoc_legendre(L, np.cos(th), np.sin(th))
    Pp = oracle.assoc_legendre(L, np.cos(th + h), np.sin(th + h))
    Pm = oracle.assoc_legendre(L, np.cos(th - h), np.sin(th - h))
    fd = (Pp - Pm) / (2 * h)
    dP = oracle.dlegendre_dtheta(P)
    scale = np.abs(dP).max(axis=-1, keepdims=True) + 1e-300
    assert np.all(np.abs(dP - fd) <= 1e-7 * scale)
    Q = oracle.legendre_m_over_sin(P)
    m = np.arange(L + 1)[None, :, None]
    direct = m * P / np.sin(th)[None, None, :]
    assert np.allclose(Q, direct, rtol=1e-11, atol=1e-11 * np.abs(direct).max())
    # at the pole: only m = 1 survives, m P_l^1 / sin -> -l(l+1)/2 at theta = 0
    P0 = oracle.assoc_legendre(L, np.array([1.0]), np.array([0.0]))
    Q0 = oracle.legendre_m_over_sin(P0)
    for l in range(1, L + 1):
        assert Q0[l, 1, 0] == pytest.approx(-l * (l + 1) / 2, rel=1e-14)
        assert np.all(Q0[l, 2:, 0] == 0.0)


# ---------------------------------------------------------------------------
# Cell integrals of §2 and the Appendix
# ---------------------------------------------------------------------------

def test_polar_integrals_against_high_precision_quadrature():
    """Eq. tlm evaluated independently at 20 digits (mpmath's Ferrers function,
    which carries the same Condon-Shortley phase) on cells of the three grids."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 20
    rng = np.random.default_rng(21)
    for name in ("tiny", "mid", "production"):
        spec = inputs.GRIDS[name]()
        te, _ = oracle.angular_edges(spec.n_theta, spec.n_phi, spec.delta_theta, spec.delta_phi)
        T = oracle.polar_integrals(30, te)
        for _ in range(3):
            j = int(rng.integers(spec.n_theta))
            l = int(rng.integers(0, 31))
            m = int(rng.integers(0, l + 1))
            ref = mpmath.quad(lambda t: mpmath.sin(t) * mpmath.legenp(l, m, mpmath.cos(t), type=2),
                              [mpmath.mpf(te[j]), mpmath.mpf(te[j + 1])], method="gauss-legendre")
            t, w = _gl(te[j], te[j + 1], 64)
            size = np.sum(w * np.abs(np.sin(t) * special.lpmv(m, l, np.cos(t))))
            assert abs(T[l, m, j] - float(ref)) <= 1e-13 * size, (name, j, l, m)


@pytest.mark.parametrize("name,lmax,diag_tol", [("tiny", 8, 1e-12), ("mid", 15, 1e-12),
                                                ("production", 25, 1e-10)])
def test_appendix_recurrences_agree_with_definition(name, lmax, diag_tol):
    """The paper's recurrences (printed order, reading R1) against Eq. tlm.
    Off the diagonal they agree to rounding; the T^(ll) diagonal carries the
    amplified rounding of reading R8."""
    spec = inputs.GRIDS[name]()
    te, _ = oracle.angular_edges(spec.n_theta, spec.n_phi, spec.delta_theta, spec.delta_phi)
    T = oracle.polar_integrals(lmax, te)
    Ta = oracle.polar_integrals_appendix(lmax, te)
    # scale: int |sin P_l^m| over the cell, computed with the same rule
    nodes, weights = npleg.leggauss(lmax + 32)
    for j in range(spec.n_theta):
        half = 0.5 * (te[j + 1] - te[j])
        t = 0.5 * (te[j] + te[j + 1]) + half * nodes
        P = oracle.assoc_legendre(lmax, np.cos(t), np.sin(t))
        size = np.abs(P * np.sin(t)) @ (half * weights) + 1e-300
        err = np.abs(T[:, :, j] - Ta[:, :, j]) / size
        for l in range(lmax + 1):
            assert err[l, :l].max(initial=0.0) <= 1e-12, (j, l)
            assert err[l, l] <= diag_tol, (j, l)


def _golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def test_polar_integrals_full_range_closed_forms():
    # cells tiling [0, pi]; sums over cells are integrals of P_l^m over [-1, 1]
    te = np.linspace(0.0, math.pi, 37)
    T = oracle.polar_integrals(12, te).sum(axis=-1)
    Ta = oracle.polar_integrals_appendix(12, te).sum(axis=-1)
    for l, m, val in _golden("full_range_polar_integrals.txt"):
        l, m, val = int(l), int(m), float(val)
        assert T[l, m] == pytest.approx(val, rel=1e-13, abs=1e-13), (l, m)
        assert Ta[l, m] == pytest.approx(val, rel=1e-13, abs=1e-13), (l, m)
    for l in range(1, 13):
        assert abs(T[l, 0]) <= 1e-13                      # int P_l = 0, l > 0


@pytest.mark.parametrize("th_lo, th_hi, n", [(math.pi / 4 - 0.03, 3 * math.pi / 4 + 0.03, 90),
                                             (math.pi / 4 - 0.03, 3 * math.pi / 4 + 0.03, 17),
                                             (0.0, math.pi, 45)])
def test_equatorial_parity_of_legendre_tables(th_lo, th_hi, n):
    """Grids symmetric about the equator (the Yin-Yang patch, the full polar
    grid; odd n has a middle cell that is its own mirror): under
    theta -> pi - theta, P_l^m(cos theta), m P_l^m / sin theta and the cell
    integrals T_j change sign by (-1)^(l+m), dP/dtheta by the opposite sign.
    The float64 polar stages of the GPU path sum half the rows on this."""
    lmax = 25
    edges = np.linspace(th_lo, th_hi, n + 1)
    th = 0.5 * (edges[1:] + edges[:-1])
    P = yinyang.assoc_legendre(lmax, np.cos(th), np.sin(th))
    tables = {"P": (P, 0), "dP": (yinyang.dlegendre_dtheta(P), 1), "mP/sin": (yinyang.legendre_m_over_sin(P), 0),
              "T": (oracle.polar_integrals(lmax, edges), 0)}
    for name, (tab, flip) in tables.items():
        for l in range(lmax + 1):
            for m in range(l + 1):
                row = tab[l, m]
                scale = np.abs(row).max()
                if scale == 0.0:
                    continue
                sign = (-1) ** (l + m + flip)
                assert np.abs(row[::-1] - sign * row).max() <= 1e-12 * scale, (name, l, m)


def test_T22_reading_R1():
    # printed seed (literal) vs bracketed seed vs the T^(ll) recurrence at l = 2
    tm, tp = 0.0, math.pi
    literal = 0.25 * (math.cos(3 * tp) - math.cos(3 * tm)) - 9 * (math.cos(tp) - math.cos(tm))
    bracketed = 0.25 * ((math.cos(3 * tp) - math.cos(3 * tm)) - 9 * (math.cos(tp) - math.cos(tm)))
    assert literal == pytest.approx(17.5)
    assert bracketed == pytest.approx(4.0)                 # int_0^pi 3 sin^3 = 4
    te = np.array([0.3, 0.7, 1.9])
    T = oracle.polar_integrals_appendix(2, te)
    x = np.cos(te)
    rec = (x[:-1] * 3 * (1 - x[:-1] ** 2) - x[1:] * 3 * (1 - x[1:] ** 2) + 6 * (x[:-1] - x[1:])) / 3
    assert np.allclose(T[2, 2], rec, rtol=1e-14)


@pytest.mark.parametrize("name", ["tiny", "production"])
def test_azimuthal_integrals_against_quadrature(name):
    spec = inputs.GRIDS[name]()
    _, pe = oracle.angular_edges(spec.n_theta, spec.n_phi, spec.delta_theta, spec.delta_phi)
    L = 40
    C, S = oracle.azimuthal_integrals(L, pe)
    for k in range(0, spec.n_phi, 7):
        p, w = _gl(pe[k], pe[k + 1], 60)
        for m in range(L + 1):
            assert C[m, k] == pytest.approx(np.sum(w * np.cos(m * p)), abs=1e-15)
            assert S[m, k] == pytest.approx(np.sum(w * np.sin(m * p)), abs=1e-15)


def test_azimuthal_full_circle():
    pe = np.linspace(-math.pi, math.pi, 91)
    C, S = oracle.azimuthal_integrals(20, pe)
    assert C[0].sum() == pytest.approx(2 * math.pi, rel=1e-15)
    assert np.all(np.abs(C[1:].sum(axis=1)) < 1e-13)
    assert np.all(np.abs(S.sum(axis=1)) < 1e-13)


def test_radial_integrals_against_quadrature():
    r = np.logspace(-4, 0, 41)
    L = 40
    Rin, Rout = oracle.radial_integrals(L, r)
    for i in range(r.size - 1):
        x, w = _gl(r[i], r[i + 1], 40)
        for l in range(L + 1):
            ref_in = np.sum(w * x ** (l + 2))
            ref_out = np.sum(w * x ** (1 - l))
            assert Rin[l, i] == pytest.approx(ref_in, rel=1e-11)
            assert Rout[l, i] == pytest.approx(ref_out, rel=1e-11)
    # the l = 2 case is the logarithm
    assert Rout[2, 3] == pytest.approx(math.log(r[4] / r[3]), rel=1e-14)


# ---------------------------------------------------------------------------
# §4 geometry
# ---------------------------------------------------------------------------

def test_transform_is_involution_and_matches_cartesian_map():
    rng = np.random.default_rng(5)
    th = rng.uniform(0.05, math.pi - 0.05, 500)
    ph = rng.uniform(-math.pi, math.pi, 500)
    t2, p2 = oracle.other_patch_angles(th, ph)
    t3, p3 = oracle.other_patch_angles(t2, p2)
    assert np.allclose(t3, th, atol=1e-12)
    assert np.allclose(np.cos(p3 - ph), 1.0, atol=1e-12)
    v = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    w = oracle.other_patch_cartesian(v)
    u = np.stack([np.sin(t2) * np.cos(p2), np.sin(t2) * np.sin(p2), np.cos(t2)])
    assert np.allclose(w, u, atol=1e-12)
    M = oracle.other_patch_cartesian(np.eye(3))
    assert np.linalg.det(M) == pytest.approx(1.0)
    assert np.allclose(M @ M, np.eye(3))


def _domain_indicator(theta, phi, spec):
    """Is the point (own-patch angles) inside the other patch's domain?  Uses
    the transform and the other patch's interval bounds directly."""
    t2, p2 = oracle.other_patch_angles(theta, phi)
    return ((t2 >= math.pi / 4 - spec.delta_theta) & (t2 <= 3 * math.pi / 4 + spec.delta_theta)
            & (p2 >= -3 * math.pi / 4 - spec.delta_phi) & (p2 <= 3 * math.pi / 4 + spec.delta_phi))


@pytest.mark.parametrize("name", ["tiny", "mid", "production"])
def test_weights_two_pi_identity(name, oracle_grid):
    spec = inputs.GRIDS[name]()
    g = oracle_grid(spec)
    te, pe = g.theta_edges, g.phi_edges
    dO = (np.cos(te[:-1]) - np.cos(te[1:]))[:, None] * (pe[1:] - pe[:-1])[None, :]
    two_pi = float(_golden("weight_identity.txt")[0][1])
    assert abs((dO * g.w).sum() - two_pi) <= 1e-12
    assert g.w.min() >= 0.5 - 1e-14 and g.w.max() <= 1.0 + 1e-14
    # symmetric under phi -> -phi and theta -> pi - theta
    assert np.allclose(g.w, g.w[:, ::-1], atol=1e-13)
    assert np.allclose(g.w, g.w[::-1, :], atol=1e-13)


@pytest.mark.parametrize("dt,dp", [(0.0, 0.0), (0.05, 0.02), (0.1, 0.13)])
def test_weights_identity_other_buffers(dt, dp):
    te, pe = oracle.angular_edges(20, 60, dt, dp)
    w = oracle.overlap_weights(te, pe, dt, dp)
    dO = (np.cos(te[:-1]) - np.cos(te[1:]))[:, None] * (pe[1:] - pe[:-1])[None, :]
    assert abs((dO * w).sum() - 2 * math.pi) <= 1e-12


def test_weights_cut_cells_against_sampling(oracle_grid):
    spec = inputs.tiny_grid()
    g = oracle_grid(spec)
    te, pe = g.theta_edges, g.phi_edges
    ns = 400
    # u-grid uniform in cos(theta) so samples are equal-area
    checked = 0
    for j in range(spec.n_theta):
        for k in range(spec.n_phi):
            ct = np.cos(te[j]) + (np.cos(te[j + 1]) - np.cos(te[j])) * (np.arange(ns) + 0.5) / ns
            ph = pe[k] + (pe[k + 1] - pe[k]) * (np.arange(ns) + 0.5) / ns
            T, P = np.meshgrid(np.arccos(ct), ph, indexing="ij")
            frac = _domain_indicator(T, P, spec).mean()
            assert abs((1 - 0.5 * frac) - g.w[j, k]) <= 2.0 / ns, (j, k)
            checked += 0 < frac < 1
    assert checked > 20


def test_weights_deep_overlap_and_exterior(oracle_grid):
    spec = inputs.mid_grid()
    g = oracle_grid(spec)
    # the patch corner (theta = pi/4, phi = 3pi/4 + ...) lies in the overlap; the
    # cell at the equator, phi = 0 lies only in its own patch
    j0 = 0
    k_mid = spec.n_phi // 2
    assert g.w[spec.n_theta // 2, k_mid] == 1.0
    assert g.w[j0, 0] == pytest.approx(0.5, abs=1e-14)


# ---------------------------------------------------------------------------
# §5 spherical test and the brute-force discrete sum
# ---------------------------------------------------------------------------

def _shell_closed_form(r_edges, rho_shell, G):
    """Phi(r_n^+) of a shell-piecewise-constant density (shell theorem):
    -G [M(<r)/r + 4 pi sum_{i>n} rho_i (r_i+^2 - r_i-^2)/2]."""
    rm, rp = r_edges[:-1], r_edges[1:]
    M = np.cumsum(4 * math.pi / 3 * rho_shell * (rp ** 3 - rm ** 3))
    outer = 2 * math.pi * rho_shell * (rp ** 2 - rm ** 2)
    out_sum = np.concatenate([np.cumsum(outer[::-1])[::-1][1:], [0.0]])
    return -G * (M / rp + out_sum), -G * M / rp ** 2


@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_monopole_exact_for_spherical_density(name):
    spec = inputs.GRIDS[name]()
    rng = np.random.default_rng(7)
    rho_shell = rng.uniform(0.1, 2.0, spec.n_r)
    g = oracle.OracleGrid(spec.r_edges, spec.n_theta, spec.n_phi, spec.delta_theta,
                          spec.delta_phi, 0, G=2.5)
    rho = np.broadcast_to(rho_shell[:, None, None], (spec.n_r, spec.n_theta, spec.n_phi))
    res = g.solve(rho, rho, gradient=True)
    phi_ref, g_ref = _shell_closed_form(spec.r_edges, rho_shell, 2.5)
    for q in ("yin", "yang"):
        assert np.abs(res["phi_" + q] - phi_ref[:, None, None]).max() <= 1e-12 * np.abs(phi_ref).max()
        gr = res["grad_" + q]
        assert np.abs(gr[0] - g_ref[:, None, None]).max() <= 1e-12 * np.abs(g_ref).max()
        assert np.abs(gr[1:]).max() <= 1e-12 * np.abs(g_ref).max()


def test_centred_uniform_sphere_inside_and_outside():
    # R = r_edges[20] on an interface; the ball r < r_edges[0] is empty (R5)
    spec = inputs.tiny_grid()
    R = spec.r_edges[20]
    rho_shell = np.where(spec.r_edges[1:] <= R, 1.0, 0.0)
    g = oracle.OracleGrid(spec.r_edges, spec.n_theta, spec.n_phi, spec.delta_theta,
                          spec.delta_phi, 0)
    rho = np.broadcast_to(rho_shell[:, None, None], (spec.n_r, spec.n_theta, spec.n_phi))
    phi = g.solve(rho, rho)["phi_yin"][:, 0, 0]
    r = spec.r_edges[1:]
    r0 = spec.r_edges[0]
    M = 4 * math.pi / 3 * (R ** 3 - r0 ** 3)
    ref = np.where(r <= R, -(4 * math.pi / 3 * (r ** 3 - r0 ** 3) / r + 2 * math.pi * (R ** 2 - r ** 2)),
                   -M / r)
    assert np.abs(phi - ref).max() <= 1e-12 * np.abs(ref).max()
    # the continuum form -G M (3R^2 - r^2) / (2R^3) (r0 -> 0) differs from the
    # discretised one by the empty ball only: G (4 pi / 3) r0^3 / r
    inside = r <= R
    M0 = 4 * math.pi / 3 * R ** 3
    cont = -M0 * (3 * R ** 2 - r ** 2) / (2 * R ** 3)
    empty = 4 * math.pi / 3 * r0 ** 3 / r
    assert np.abs(phi[inside] - cont[inside] - empty[inside]).max() <= 1e-12 * np.abs(cont).max()


def test_spherical_leakage_small_and_decreasing():
    # l > 0 leakage of a spherical density comes only from cut-cell averaging of w
    errs = []
    for n_t, n_p in ((12, 36), (24, 72)):
        r_edges = np.logspace(-2, 0, 9)
        g = oracle.OracleGrid(r_edges, n_t, n_p, 0.0, 0.0, 6)
        rho = np.ones((8, n_t, n_p))
        res = g.solve(rho, rho)
        ref, _ = _shell_closed_form(r_edges, np.ones(8), 1.0)
        errs.append(np.abs(res["phi_yin"] - ref[:, None, None]).max() / np.abs(ref).max())
    assert errs[0] < 1e-2
    assert errs[1] < errs[0]


def _random_targets(spec, n, seed):
    rng = np.random.default_rng(seed)
    return [(("yin", "yang")[int(rng.integers(2))], int(rng.integers(spec.n_r)),
             int(rng.integers(spec.n_theta)), int(rng.integers(spec.n_phi))) for _ in range(n)]


def test_bruteforce_addition_theorem_tiny(oracle_grid):
    """Whole discrete formula (normalisations, T/C/S, cross-patch evaluation,
    gradient basis rotation) against the addition-theorem brute force."""
    spec = inputs.tiny_grid()
    g = oracle_grid(spec)
    ry, rg = inputs.tiny_density(spec)
    res = g.solve(ry, rg, gradient=True)
    targets = _random_targets(spec, 24, 11)
    phi_bf, g_bf = bf.potential_and_gradient(spec, g.w, {"yin": ry, "yang": rg}, targets)
    phi_o = np.array([res["phi_" + p][n, j, k] for p, n, j, k in targets])
    g_o = np.array([res["grad_" + p][:, n, j, k] for p, n, j, k in targets])
    assert np.abs(phi_bf - phi_o).max() <= 1e-12 * np.abs(phi_o).max()
    assert np.abs(g_bf - g_o).max() <= 1e-12 * np.abs(g_o).max()


def test_bruteforce_random_density_odd_buffers():
    """Same brute-force pin on a random density, unequal buffers and l_max = 5."""
    spec = inputs.GridSpec("odd", np.linspace(0.0, 1.0, 7), 10, 26, 0.07, 0.11, 5, 0.7)
    g = oracle.OracleGrid(spec.r_edges, spec.n_theta, spec.n_phi, spec.delta_theta,
                          spec.delta_phi, spec.lmax, spec.G)
    rng = np.random.default_rng(12)
    ry = rng.uniform(0, 1, (6, 10, 26))
    rg = rng.uniform(0, 1, (6, 10, 26))
    res = g.solve(ry, rg, gradient=True)
    targets = _random_targets(spec, 16, 13)
    phi_bf, g_bf = bf.potential_and_gradient(spec, g.w, {"yin": ry, "yang": rg}, targets)
    phi_o = np.array([res["phi_" + p][n, j, k] for p, n, j, k in targets])
    g_o = np.array([res["grad_" + p][:, n, j, k] for p, n, j, k in targets])
    assert np.abs(phi_bf - phi_o).max() <= 1e-12 * np.abs(phi_o).max()
    assert np.abs(g_bf - g_o).max() <= 1e-12 * np.abs(g_o).max()


def test_green_function_convergence_with_lmax():
    """The truncated expansion approaches the exact 1/|x-x'| sum as l_max grows."""
    spec0 = inputs.GridSpec("g", np.linspace(0.05, 1.0, 9), 12, 36, 0.0, 0.0, 1)
    rng = np.random.default_rng(14)
    ry = rng.uniform(0.5, 1.5, (8, 12, 36))
    rg = rng.uniform(0.5, 1.5, (8, 12, 36))
    targets = [("yin", 7, 3, 10), ("yang", 7, 8, 20), ("yin", 2, 6, 30)]
    errs = []
    w = None
    for L in (1, 4, 10):
        g = oracle.OracleGrid(spec0.r_edges, 12, 36, 0.0, 0.0, L)
        w = g.w
        res = g.solve(ry, rg)
        errs.append(np.array([res["phi_" + p][n, j, k] for p, n, j, k in targets]))
    exact = bf.green_potential(spec0, w, {"yin": ry, "yang": rg}, targets)
    e = [np.abs(x - exact).max() / np.abs(exact).max() for x in errs]
    assert e[2] < e[1] < e[0]
    assert e[2] < 1e-2


def test_offcentre_sphere_point_mass_limit(oracle_grid):
    """Outside r > |c| + a an off-centre sphere has the moments of a point mass;
    the oracle with the tiny grid approaches -GM/|x - c| there (sampling error
    of the cell averages only)."""
    spec = inputs.tiny_grid()
    g = oracle_grid(spec)
    c = np.array([0.2, 0.1, -0.15])
    a = 0.1
    ry, rg = inputs.offcentre_sphere_density(spec, c, a, 5.0)
    res = g.solve(ry, rg)
    M = 5.0 * 4 * math.pi / 3 * a ** 3
    r = spec.r_edges[1:]
    n_out = np.nonzero(r > 1.6 * (np.linalg.norm(c) + a))[0]
    th, ph = g.target_theta, g.target_phi
    u = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    for n in n_out:
        x = r[n] * u
        exact = -M / np.linalg.norm(x - c[:, None], axis=0)
        rel = np.abs(res["phi_yin"][n].reshape(-1) - exact).max() / np.abs(exact).max()
        assert rel < 2e-2


# ---------------------------------------------------------------------------
# symmetries and linearity
# ---------------------------------------------------------------------------

def test_swap_symmetry_bitwise(oracle_grid):
    spec = inputs.tiny_grid()
    g = oracle_grid(spec)
    ry, rg = inputs.tiny_density(spec)
    a = g.solve(ry, rg, gradient=True)
    b = g.solve(rg, ry, gradient=True)
    assert np.array_equal(a["phi_yin"], b["phi_yang"])
    assert np.array_equal(a["phi_yang"], b["phi_yin"])
    assert np.array_equal(a["grad_yin"], b["grad_yang"])


def test_linearity(oracle_grid):
    spec = inputs.tiny_grid()
    g = oracle_grid(spec)
    rng = np.random.default_rng(15)
    shape = (spec.n_r, spec.n_theta, spec.n_phi)
    r1 = [rng.uniform(0, 1, shape) for _ in range(2)]
    r2 = [rng.uniform(0, 1, shape) for _ in range(2)]
    a = g.solve(*r1)["phi_yin"]
    b = g.solve(*r2)["phi_yin"]
    c = g.solve(2 * r1[0] - 3 * r2[0], 2 * r1[1] - 3 * r2[1])["phi_yin"]
    assert np.abs(c - (2 * a - 3 * b)).max() <= 1e-13 * np.abs(c).max()


def test_gradient_matches_finite_differences_in_angle(oracle_grid):
    spec = inputs.mid_grid()
    spec = inputs.GridSpec("fd", spec.r_edges[::10], 45, 135, 0.0, 0.0, 10)
    g = oracle_grid(spec)
    ry, rg = inputs.oblate_density(inputs.GridSpec("fd", spec.r_edges, 45, 135, 0.0, 0.0, 10))
    coef = g.radial_sums(*g.analysis(rg))
    rng = np.random.default_rng(16)
    th = rng.uniform(0.3, 2.8, 20)
    ph = rng.uniform(-3.0, 3.0, 20)
    h = 1e-5
    v = g.evaluate_gradient(coef, th, ph)
    _, e_t, e_p = yinyang.spherical_basis(th, ph)
    dth = (g.evaluate(coef, th + h, ph) - g.evaluate(coef, th - h, ph)) / (2 * h)
    dph = (g.evaluate(coef, th, ph + h) - g.evaluate(coef, th, ph - h)) / (2 * h)
    r = spec.r_edges[1:][:, None]
    g_t = np.einsum("cnp,cp->np", v, e_t)
    g_p = np.einsum("cnp,cp->np", v, e_p)
    assert np.abs(g_t + dth / r).max() <= 1e-6 * np.abs(g_t).max()
    assert np.abs(g_p + dph / (r * np.sin(th))).max() <= 1e-6 * np.abs(g_p).max()


# ---------------------------------------------------------------------------
# §2: the full spherical polar grid (one patch, w = 1; reading R10)
# ---------------------------------------------------------------------------

def test_polar_grid_spherical_density_exact_at_any_lmax():
    """Over the whole sphere the cell integrals of every l > 0 harmonic sum to
    zero (T over [0, pi] times C/S over [0, 2 pi)), so a spherical density
    gives the shell closed form at any l_max, with no leakage."""
    spec = inputs.tiny_polar_grid()
    rng = np.random.default_rng(21)
    rho_shell = rng.uniform(0.1, 2.0, spec.n_r)
    g = oracle.OraclePolarGrid(spec.r_edges, spec.n_theta, spec.n_phi, 8, G=1.7)
    rho = np.broadcast_to(rho_shell[:, None, None], (spec.n_r, spec.n_theta, spec.n_phi))
    res = g.solve(rho, gradient=True)
    phi_ref, g_ref = _shell_closed_form(spec.r_edges, rho_shell, 1.7)
    assert np.abs(res["phi"] - phi_ref[:, None, None]).max() <= 1e-12 * np.abs(phi_ref).max()
    assert np.abs(res["grad"][0] - g_ref[:, None, None]).max() <= 1e-12 * np.abs(g_ref).max()
    assert np.abs(res["grad"][1:]).max() <= 1e-12 * np.abs(g_ref).max()


def test_polar_grid_cells_tile_the_sphere():
    g = oracle.OraclePolarGrid(np.linspace(0.0, 1.0, 3), 7, 13, 2)
    assert g.theta_edges[0] == 0.0 and abs(g.theta_edges[-1] - math.pi) <= 1e-15
    assert g.phi_edges[0] == 0.0 and abs(g.phi_edges[-1] - 2 * math.pi) <= 1e-15
    dO = np.outer(np.cos(g.theta_edges[:-1]) - np.cos(g.theta_edges[1:]), np.diff(g.phi_edges))
    assert abs(dO.sum() - 4 * math.pi) <= 1e-13
    assert np.all(g.w == 1.0)


def test_polar_grid_bruteforce_addition_theorem():
    """Whole discrete formula on the polar grid against the brute-force sum
    through the addition theorem, on a random density."""
    spec = inputs.polar_grid(np.linspace(0.0, 1.0, 7), 10, 22, 6, G=0.8)
    g = oracle.OraclePolarGrid(spec.r_edges, spec.n_theta, spec.n_phi, spec.lmax, spec.G)
    rng = np.random.default_rng(22)
    rho = rng.uniform(0, 1, (6, 10, 22))
    res = g.solve(rho, gradient=True)
    targets = [("yin", int(rng.integers(6)), int(rng.integers(10)), int(rng.integers(22))) for _ in range(16)]
    phi_bf, g_bf = bf.potential_and_gradient(spec, g.w, {"yin": rho}, targets)
    phi_o = np.array([res["phi"][n, j, k] for _, n, j, k in targets])
    g_o = np.array([res["grad"][:, n, j, k] for _, n, j, k in targets])
    assert np.abs(phi_bf - phi_o).max() <= 1e-12 * np.abs(phi_o).max()
    assert np.abs(g_bf - g_o).max() <= 1e-12 * np.abs(g_o).max()


def test_polar_grid_green_function_convergence_with_lmax():
    """The truncated expansion on the polar grid approaches the exact
    1/|x - x'| sum as l_max grows."""
    spec = inputs.polar_grid(np.linspace(0.05, 1.0, 9), 12, 24, 1)
    rng = np.random.default_rng(23)
    rho = rng.uniform(0.5, 1.5, (8, 12, 24))
    targets = [("yin", 7, 3, 10), ("yin", 7, 8, 20), ("yin", 2, 6, 3)]
    errs = []
    for L in (1, 4, 10):
        res = oracle.OraclePolarGrid(spec.r_edges, 12, 24, L).solve(rho)
        errs.append(np.array([res["phi"][n, j, k] for _, n, j, k in targets]))
    exact = bf.green_potential(spec, np.ones((12, 24)), {"yin": rho}, targets)
    e = [np.abs(x - exact).max() / np.abs(exact).max() for x in errs]
    assert e[2] < e[1] < e[0]
    assert e[2] < 1e-2
