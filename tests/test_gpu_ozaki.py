"""YY_FP64_OZAKI: float64 results with the synthesis's azimuthal stage on the
tensor cores by the Ozaki scheme, against the float64 oracle and against
the CUDA-core float64 path.  The float64 bar is 1e-12 relative (Phi
pointwise, -grad Phi normwise); the tests assert 4e-13 against the oracle,
about 4.6x the worst error measured (8.6e-14), so that a regression shows
before the bar is reached.

Each operand is six balanced base-256 digits of round(|x| 2^48) under a
per-row scale that puts |x| at most 1/2, so a product term is off by at most
2^-49 of the scales (2^-46 of the largest |G|), with a rounding error of
either sign; over K <= 63 terms that is about sqrt(K / 3) 2^-46 of the row's
largest value, 7e-14 at K = 51.  2e-13 relative is the bar against the
CUDA-core float64 path.
"""

import numpy as np
import pytest

from paper_1806_04593_gb300 import inputs

from .gpu_common import field_err, gpu_solve, grad_err, lib, phi_err, require_gpu

pytestmark = pytest.mark.gpu

TOL_FP64 = 4e-13
TOL_VS_FP64_PATH = 2e-13


@pytest.fixture(scope="module")
def yy():
    require_gpu()
    return lib()


_GRIDS = {}


def _grid(yy, spec):
    if spec.name not in _GRIDS:
        g = yy.Grid.from_spec(spec)
        g.prepare("fp64_ozaki")
        _GRIDS[spec.name] = g
    return _GRIDS[spec.name]


@pytest.mark.parametrize("analysis", ["auto", "dense"])
@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_ozaki_matches_oracle_and_fp64_path(yy, oracle_grid, name, analysis):
    spec = inputs.GRIDS[name]()
    g = _grid(yy, spec)
    ry, rg = inputs.density_for(spec)
    g.set_analysis(analysis)
    try:
        oz = gpu_solve(g, ry, rg, gradient=True, prec="fp64_ozaki")
        n_oz = yy.yy_last_launch_count(g.handle)
        f64 = gpu_solve(g, ry, rg, gradient=True, prec="fp64")
        n_64 = yy.yy_last_launch_count(g.handle)
    finally:
        g.set_analysis("auto")
    assert yy.yy_last_device_status(g.handle) == yy.YY_OK
    if analysis == "auto":
        # separable both ways; the emulated analysis launches one kernel more
        # (the digit rows) than its float64 counterpart, the synthesis two
        # (the coefficients as fp32 pairs, the digit products)
        assert n_oz == n_64 + 3, (n_oz, n_64)
    ref = oracle_grid(spec).solve(ry, rg, gradient=True)
    for q in ("yin", "yang"):
        assert phi_err(oz["phi_" + q], ref["phi_" + q]) <= TOL_FP64, q
        assert grad_err(oz["grad_" + q], ref["grad_" + q]) <= TOL_FP64, q
    for key in oz:
        assert field_err(key, oz[key], f64[key]) <= TOL_VS_FP64_PATH, key


def test_ozaki_production_sampled(yy, oracle_grid):
    spec = inputs.production_grid()
    g = _grid(yy, spec)
    ry, rg = inputs.density_for(spec)
    out = gpu_solve(g, ry, rg, gradient=True, prec="fp64_ozaki")
    assert yy.yy_last_device_status(g.handle) == yy.YY_OK
    rng = np.random.default_rng(44)
    cells = np.sort(rng.choice(spec.n_ang, 64, replace=False))
    ref = oracle_grid(spec).solve(ry, rg, gradient=True, cells=cells)
    j, k = np.divmod(cells, spec.n_phi)
    for q in ("yin", "yang"):
        assert phi_err(out["phi_" + q][:, j, k], ref["phi_" + q]) <= TOL_FP64
        assert grad_err(out["grad_" + q][:, :, j, k], ref["grad_" + q]) <= TOL_FP64


def test_ozaki_analysis_in_several_fills(yy, oracle_grid):
    """Rows of 600 longitudes: the emulated analysis adds four fills of up to
    160; against the oracle on sampled cells and the float64 path on all."""
    import torch
    spec = inputs.polar_grid(np.logspace(-3, 0, 31), 60, 600, 12, "polar_600_oz")
    g = yy.Grid.from_spec(spec)
    try:
        g.prepare("fp64_ozaki")
        rho, _ = inputs.pns_density(spec, 8, 0.05)
        r = torch.as_tensor(np.ascontiguousarray(rho), device="cuda")
        out = g.solve(r, gradient=True, prec="fp64_ozaki")
        torch.cuda.synchronize()
        n_oz = yy.yy_last_launch_count(g.handle)
        f64 = g.solve(r, gradient=True, prec="fp64")
        torch.cuda.synchronize()
        assert yy.yy_last_device_status(g.handle) == yy.YY_OK
        # polar grid: emulated analysis (digit rows, digit products, polar
        # stage), scans, synthesis (coefficient pairs, polar stage, digit
        # products)
        assert n_oz == 7, n_oz
        for key in ("phi", "grad"):
            assert field_err(key, out[key].cpu().numpy(), f64[key].cpu().numpy()) <= TOL_VS_FP64_PATH, key
        rng = np.random.default_rng(48)
        cells = np.sort(rng.choice(spec.n_ang, 48, replace=False))
        ref = oracle_grid(spec).solve(rho, gradient=True, cells=cells)
        j, k = np.divmod(cells, spec.n_phi)
        assert phi_err(out["phi"].cpu().numpy()[:, j, k], ref["phi"]) <= TOL_FP64
        assert grad_err(out["grad"].cpu().numpy()[:, :, j, k], ref["grad"]) <= TOL_FP64
    finally:
        g.close()


def test_ozaki_ragged_and_highest_degree(yy):
    """Sizes that are multiples of no tile (17 x 41 cells, 131 zones; an odd
    n_theta, whose middle polar row is its own mirror in the polar synthesis
    stage); l_max = 31, the last in G rows of 64 slots (no room for the bias
    columns: the general synthesis kernel); l_max = 40 and 63, in rows of 128
    slots (the polar stage's second slot group, the analysis in tiles of 32
    slots), 63 the largest."""
    from oracle import OracleGrid
    for n_r, nt, npp, lmax, seed in ((131, 17, 41, 13, 45), (40, 20, 60, 31, 46), (36, 22, 66, 40, 47),
                                     (20, 24, 70, 63, 48)):
        spec = inputs.GridSpec(f"ragged_oz_{lmax}", np.logspace(-2, 0, n_r + 1), nt, npp, 0.03, 0.05, lmax, 1.0)
        rng = np.random.default_rng(seed)
        ry = rng.uniform(0.5, 1.5, (n_r, nt, npp))
        rg = rng.uniform(0.5, 1.5, (n_r, nt, npp))
        g = yy.Grid.from_spec(spec)
        try:
            g.prepare("fp64_ozaki")
            out = gpu_solve(g, ry, rg, gradient=True, prec="fp64_ozaki")
            assert yy.yy_last_device_status(g.handle) == yy.YY_OK
        finally:
            g.close()
        ref = OracleGrid(spec.r_edges, nt, npp, 0.03, 0.05, lmax).solve(ry, rg, gradient=True)
        for q in ("yin", "yang"):
            assert phi_err(out["phi_" + q], ref["phi_" + q]) <= TOL_FP64, (lmax, q)
            assert grad_err(out["grad_" + q], ref["grad_" + q]) <= TOL_FP64, (lmax, q)


def test_ozaki_lowest_degrees(yy):
    """l_max = 0 (the monopole alone: one slot and one polar order, the polar
    stage's loads past the degree-0 coefficient row landing in the spare rows
    after the last field), 1 and 2, against the oracle."""
    from oracle import OracleGrid
    for lmax, seed in ((0, 51), (1, 52), (2, 53)):
        spec = inputs.GridSpec(f"oz_low_{lmax}", np.logspace(-2, 0, 10), 12, 36, 0.03, 0.05, lmax, 1.0)
        rng = np.random.default_rng(seed)
        ry = rng.uniform(0.5, 1.5, (9, 12, 36))
        rg = rng.uniform(0.5, 1.5, (9, 12, 36))
        g = yy.Grid.from_spec(spec)
        try:
            g.prepare("fp64_ozaki")
            out = gpu_solve(g, ry, rg, gradient=True, prec="fp64_ozaki")
            assert yy.yy_last_device_status(g.handle) == yy.YY_OK
        finally:
            g.close()
        ref = OracleGrid(spec.r_edges, 12, 36, 0.03, 0.05, lmax).solve(ry, rg, gradient=True)
        for q in ("yin", "yang"):
            assert phi_err(out["phi_" + q], ref["phi_" + q]) <= TOL_FP64, (lmax, q)
            assert grad_err(out["grad_" + q], ref["grad_" + q]) <= TOL_FP64, (lmax, q)


def test_ozaki_polar_grid(yy, oracle_grid):
    import torch
    spec = inputs.mid_polar_grid()
    g = yy.Grid.from_spec(spec)
    try:
        g.prepare("fp64_ozaki")
        rho, _ = inputs.pns_density(spec, 3, 0.05)
        r = torch.as_tensor(np.ascontiguousarray(rho), device="cuda")
        out = g.solve(r, gradient=True, prec="fp64_ozaki")
        torch.cuda.synchronize()
        assert yy.yy_last_device_status(g.handle) == yy.YY_OK
        ref = oracle_grid(spec).solve(rho, gradient=True)
        assert phi_err(out["phi"].cpu().numpy(), ref["phi"]) <= TOL_FP64
        assert grad_err(out["grad"].cpu().numpy(), ref["grad"]) <= TOL_FP64
    finally:
        g.close()


def test_ozaki_deterministic_swap_and_zero(yy):
    spec = inputs.tiny_grid()
    g = _grid(yy, spec)
    ry, rg = inputs.density_for(spec)
    a = gpu_solve(g, ry, rg, gradient=True, prec="fp64_ozaki")
    b = gpu_solve(g, ry, rg, gradient=True, prec="fp64_ozaki")
    c = gpu_solve(g, rg, ry, gradient=True, prec="fp64_ozaki")
    for key in a:
        assert np.array_equal(a[key], b[key]), key
    assert np.array_equal(a["phi_yin"], c["phi_yang"])
    assert np.array_equal(a["grad_yang"], c["grad_yin"])
    z = np.zeros_like(ry)
    for v in gpu_solve(g, z, z, gradient=True, prec="fp64_ozaki").values():
        assert np.all(v == 0.0)


def test_ozaki_needs_prepare_and_low_degree(yy):
    import torch
    spec = inputs.tiny_grid()
    g = yy.Grid.from_spec(spec)
    try:
        x = torch.zeros((spec.n_r, spec.n_theta, spec.n_phi), dtype=torch.float64, device="cuda")
        st = yy.yy_potential(g.handle, x, x, x.clone(), x.clone(), prec=yy.YY_FP64_OZAKI)
        assert st == yy.YY_ERR_NOT_SUPPORTED
    finally:
        g.close()
    big = inputs.GridSpec("oz_lmax64", np.logspace(-2, 0, 9), 12, 36, 0.05, 0.05, 64, 1.0)   # 2 l_max + 1 > 127
    g = yy.Grid.from_spec(big)
    try:
        assert yy.yy_grid_prepare(g.handle, yy.YY_FP64_OZAKI) == yy.YY_ERR_NOT_SUPPORTED
    finally:
        g.close()


def test_ozaki_long_rows_keep_the_float64_analysis(yy, oracle_grid):
    """A grid with more than 640 longitudes (four fills of 160): the analysis
    stays float64 (one launch fewer than the emulated analysis) while the
    synthesis runs on the digits; against the oracle on sampled cells."""
    import torch
    spec = inputs.polar_grid(np.logspace(-3, 0, 41), 90, 720, 20, "polar_720_oz")
    g = yy.Grid.from_spec(spec)
    try:
        g.prepare("fp64_ozaki")
        rho, _ = inputs.pns_density(spec, 7, 0.05)
        r = torch.as_tensor(np.ascontiguousarray(rho), device="cuda")
        out = g.solve(r, gradient=True, prec="fp64_ozaki")
        torch.cuda.synchronize()
        n_oz = yy.yy_last_launch_count(g.handle)
        assert yy.yy_last_device_status(g.handle) == yy.YY_OK
        # polar grid: analysis (float64: one or two launches), scans (one),
        # synthesis (coefficient pairs, polar stage and digit products:
        # three); the emulated analysis would take three
        assert n_oz in (5, 6), n_oz
        rng = np.random.default_rng(47)
        cells = np.sort(rng.choice(spec.n_ang, 64, replace=False))
        ref = oracle_grid(spec).solve(rho, gradient=True, cells=cells)
        j, k = np.divmod(cells, spec.n_phi)
        assert phi_err(out["phi"].cpu().numpy()[:, j, k], ref["phi"]) <= TOL_FP64
        assert grad_err(out["grad"].cpu().numpy()[:, :, j, k], ref["grad"]) <= TOL_FP64
    finally:
        g.close()


@pytest.mark.parametrize("name", ["mid", "polar"])
def test_ozaki_is_homogeneous_in_the_density(yy, name):
    """The potential is linear in rho.  Every scale the Ozaki path takes
    (the digit rows' powers of two, the float-float splits' scales per
    coefficient row, per shell and per degree) follows the data, and float64
    multiplication by a power of two is exact, so rho 2^k gives exactly 2^k
    times the result: bitwise, for k = +-100 (far outside the fp32 range of
    the float-float stages).  rho 1e30 and 1e-30 stay within the float64 bar
    of the scaled result."""
    import torch
    if name == "mid":
        spec = inputs.GRIDS["mid"]()
        ry, rg = inputs.density_for(spec)
        g = _grid(yy, spec)
        solve = lambda s: gpu_solve(g, ry * s, rg * s, gradient=True, prec="fp64_ozaki")
        closer = None
    else:
        spec = inputs.mid_polar_grid()
        g = yy.Grid.from_spec(spec)
        g.prepare("fp64_ozaki")
        rho, _ = inputs.pns_density(spec, 3, 0.05)

        def solve(s):
            r = torch.as_tensor(np.ascontiguousarray(rho * s), device="cuda")
            out = g.solve(r, gradient=True, prec="fp64_ozaki")
            torch.cuda.synchronize()
            return {k: v.cpu().numpy() for k, v in out.items()}
        closer = g
    try:
        base = solve(1.0)
        assert yy.yy_last_device_status(g.handle) == yy.YY_OK
        for k in (100, -100):
            out = solve(2.0 ** k)
            assert yy.yy_last_device_status(g.handle) == yy.YY_OK
            for key in base:
                assert np.array_equal(out[key], np.ldexp(base[key], k)), (k, key)
        for s in (1e30, 1e-30):
            out = solve(s)
            for key in base:
                assert np.all(np.isfinite(out[key])), (s, key)
                assert field_err(key, out[key] / s, base[key]) <= TOL_FP64, (s, key)
    finally:
        if closer is not None:
            closer.close()


def test_ozaki_long_polar_rows_at_high_degree(yy):
    """l_max 60 on 90 polar rows: the float-float analysis stage holds more
    mirrored row pairs than its registers (45 x 121 > 8 per thread) and the
    coefficient rows (3721 of them) are longer than one shared-memory pass of
    the split, so both take their looping forms; against the CUDA-core
    float64 path on all cells."""
    import torch
    spec = inputs.polar_grid(np.logspace(-2, 0, 9), 90, 180, 60, "polar_l60_oz")
    g = yy.Grid.from_spec(spec)
    try:
        g.prepare("fp64_ozaki")
        rho, _ = inputs.pns_density(spec, 5, 0.05)
        r = torch.as_tensor(np.ascontiguousarray(rho), device="cuda")
        out = g.solve(r, gradient=True, prec="fp64_ozaki")
        torch.cuda.synchronize()
        assert yy.yy_last_device_status(g.handle) == yy.YY_OK
        f64 = g.solve(r, gradient=True, prec="fp64")
        torch.cuda.synchronize()
        for key in ("phi", "grad"):
            assert field_err(key, out[key].cpu().numpy(), f64[key].cpu().numpy()) <= TOL_VS_FP64_PATH, key
    finally:
        g.close()


def test_ozaki_polar_grid_with_odd_shell_count(yy):
    """A polar grid of 9 zones (an odd number of shells: the last block of the
    float-float analysis stage, two shells per block, has one) and 17 polar
    rows (an odd count: the middle row is its own mirror); against the
    CUDA-core float64 path on all cells."""
    import torch
    spec = inputs.polar_grid(np.logspace(-2, 0, 10), 17, 48, 11, "polar_odd_oz")
    g = yy.Grid.from_spec(spec)
    try:
        g.prepare("fp64_ozaki")
        rho, _ = inputs.pns_density(spec, 4, 0.05)
        r = torch.as_tensor(np.ascontiguousarray(rho), device="cuda")
        out = g.solve(r, gradient=True, prec="fp64_ozaki")
        torch.cuda.synchronize()
        assert yy.yy_last_device_status(g.handle) == yy.YY_OK
        f64 = g.solve(r, gradient=True, prec="fp64")
        torch.cuda.synchronize()
        for key in ("phi", "grad"):
            assert field_err(key, out[key].cpu().numpy(), f64[key].cpu().numpy()) <= TOL_VS_FP64_PATH, key
    finally:
        g.close()
