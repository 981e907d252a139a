"""GPU path (through the C ABI) against the CPU oracle.

Tolerance of the float64 path: the bar the solver is specified to is 1e-12
relative (Phi pointwise, |dPhi| / |Phi| at every cell; -grad Phi normwise);
the tests assert 1e-13, about 8x the worst error measured (1.3e-14), so
that a regression shows before the bar is reached.  Tables 1e-13.
"""

import math

import numpy as np
import pytest

from paper_1806_04593_gb300 import inputs

from .gpu_common import K_lm, field_err, gpu_solve, grad_err, lib, mode_index, phi_err, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-13


@pytest.fixture(scope="module")
def yy():
    require_gpu()
    return lib()


_GRIDS = {}


def _grid(yy, spec):
    key = spec.name
    if key not in _GRIDS:
        _GRIDS[key] = yy.Grid.from_spec(spec)
    return _GRIDS[key]


# ---------------------------------------------------------------------------
# tables
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_weight_table(yy, oracle_grid, name):
    spec = inputs.GRIDS[name]()
    g = _grid(yy, spec)
    w = g.table(yy.YY_TABLE_WEIGHTS).reshape(spec.n_theta, spec.n_phi)
    og = oracle_grid(spec)
    assert np.abs(w - og.w).max() <= 1e-13
    te, pe = og.theta_edges, og.phi_edges
    dO = (np.cos(te[:-1]) - np.cos(te[1:]))[:, None] * (pe[1:] - pe[:-1])[None, :]
    assert abs((dO * w).sum() - 2 * math.pi) <= 1e-12


def test_weight_table_production(yy, oracle_grid):
    spec = inputs.production_grid()
    g = _grid(yy, spec)
    w = g.table(yy.YY_TABLE_WEIGHTS).reshape(spec.n_theta, spec.n_phi)
    assert np.abs(w - oracle_grid(spec).w).max() <= 1e-13


@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_polar_and_analysis_tables(yy, oracle_grid, name):
    spec = inputs.GRIDS[name]()
    g = _grid(yy, spec)
    og = oracle_grid(spec)
    L = spec.lmax
    K = K_lm(og.N)
    modes = mode_index(L)
    tb = g.table(yy.YY_TABLE_TBAR).reshape(spec.n_theta, len(modes))
    ban = g.table(yy.YY_TABLE_ANALYSIS).reshape(len(modes), spec.n_ang)
    for idx, (l, m, kind) in enumerate(modes):
        ref = K[l, m] * og.T[l, m]
        assert np.abs(tb[:, idx] - ref).max() <= 1e-13 * max(np.abs(ref).max(), 1e-300), (l, m)
        cs = og.C[m] if kind == "c" else og.S[m]
        ref_b = (og.w * ref[:, None] * cs[None, :]).reshape(-1)
        scale = max(np.abs(ref_b).max(), 1e-300)
        assert np.abs(ban[idx] - ref_b).max() <= 1e-13 * scale, (l, m, kind)


@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_synthesis_tables_own_frame(yy, oracle_grid, name):
    from oracle import assoc_legendre
    spec = inputs.GRIDS[name]()
    g = _grid(yy, spec)
    og = oracle_grid(spec)
    L = spec.lmax
    K = K_lm(og.N)
    modes = mode_index(L)
    n_lm = len(modes)
    ys = g.table(yy.YY_TABLE_SYNTH).reshape(spec.n_ang, n_lm)
    th, ph = og.target_theta, og.target_phi
    P = assoc_legendre(L, np.cos(th), np.sin(th))
    for idx, (l, m, kind) in enumerate(modes):
        f = np.cos(m * ph) if kind == "c" else np.sin(m * ph)
        ref = K[l, m] * P[l, m] * f
        assert np.abs(ys[:, idx] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), (l, m, kind)


def _harmonics(L, K, modes, th, ph):
    from oracle import assoc_legendre
    P = assoc_legendre(L, np.cos(th), np.sin(th))
    out = np.empty((len(modes),) + np.shape(th))
    for idx, (l, m, kind) in enumerate(modes):
        out[idx] = K[l, m] * P[l, m] * (np.cos(m * ph) if kind == "c" else np.sin(m * ph))
    return out


@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_rotation_table_maps_other_frame_harmonics(yy, oracle_grid, name):
    """Y_i(angles in the other patch) = sum_j D^l_ij Y_j(own angles) at random
    points (oracle harmonics, oracle angle transform); D^l orthogonal and its
    own inverse (the Yin-Yang map is an involution)."""
    from oracle import other_patch_angles
    spec = inputs.GRIDS[name]()
    g = _grid(yy, spec)
    og = oracle_grid(spec)
    L = spec.lmax
    K = K_lm(og.N)
    modes = mode_index(L)
    rot = g.table(yy.YY_TABLE_ROTATION)
    assert rot.size == sum((2 * l + 1) ** 2 for l in range(L + 1))
    rng = np.random.default_rng(11)
    th = np.arccos(rng.uniform(-1.0, 1.0, 400))
    ph = rng.uniform(-math.pi, math.pi, 400)
    tx, px = other_patch_angles(th, ph)
    y_own = _harmonics(L, K, modes, th, ph)
    y_oth = _harmonics(L, K, modes, tx, px)
    for l in range(L + 1):
        w = 2 * l + 1
        off = l * (4 * l * l - 1) // 3
        D = rot[off:off + w * w].reshape(w, w)
        sl = slice(l * l, l * l + w)
        assert np.abs(D @ y_own[sl] - y_oth[sl]).max() <= 1e-12, l
        assert np.abs(D @ D.T - np.eye(w)).max() <= 1e-13, l
        assert np.abs(D @ D - np.eye(w)).max() <= 1e-13, l


# ---------------------------------------------------------------------------
# solves
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("analysis", ["separable", "dense"])
@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_fp64_potential_and_gradient_match_oracle(yy, oracle_grid, name, analysis):
    """Float64, with both analysis evaluations (separable stages and the
    dense contraction): the same moments to rounding."""
    spec = inputs.GRIDS[name]()
    g = _grid(yy, spec)
    ry, rg = inputs.density_for(spec)
    g.set_analysis(analysis)
    try:
        out = gpu_solve(g, ry, rg, gradient=True)
    finally:
        g.set_analysis("auto")
    ref = oracle_grid(spec).solve(ry, rg, gradient=True)
    for q in ("yin", "yang"):
        assert phi_err(out["phi_" + q], ref["phi_" + q]) <= TOL_FP64, q
        assert rel_l2(out["phi_" + q], ref["phi_" + q]) <= TOL_FP64, q
        assert grad_err(out["grad_" + q], ref["grad_" + q]) <= TOL_FP64, q


def test_fp64_production_sampled_cells(yy, oracle_grid):
    """Full 1-degree, l_max = 25 grid in the launch configuration of the
    benchmark; every radius at a sample of target cells."""
    spec = inputs.production_grid()
    g = _grid(yy, spec)
    ry, rg = inputs.density_for(spec)
    out = gpu_solve(g, ry, rg, gradient=True)
    rng = np.random.default_rng(31)
    cells = np.sort(rng.choice(spec.n_ang, 64, replace=False))
    ref = oracle_grid(spec).solve(ry, rg, gradient=True, cells=cells)
    j, k = np.divmod(cells, spec.n_phi)
    for q in ("yin", "yang"):
        got = out["phi_" + q][:, j, k]
        assert phi_err(got, ref["phi_" + q]) <= TOL_FP64, q
        gg = out["grad_" + q][:, :, j, k]
        assert grad_err(gg, ref["grad_" + q]) <= TOL_FP64, q


def test_fp64_separable_at_the_largest_batched_shape(yy, oracle_grid):
    """1-degree cells at l_max = 40 (the largest field of the batched
    workload): the float64 azimuthal stage runs with its short row chunk and
    the separable synthesis in row chunks, since neither's tables fit shared
    memory whole.  Sampled cells against the oracle, whole fields against the
    dense contraction."""
    spec = inputs.GridSpec("fine40", np.logspace(-3, 0, 13), 90, 270, 0.0, 0.0, 40)
    g = _grid(yy, spec)
    ry, rg = inputs.pns_density(spec, 17, 0.08)
    sep = gpu_solve(g, ry, rg, gradient=True)
    flops_sep = g.flops(True)
    g.set_analysis("dense")
    try:
        dense = gpu_solve(g, ry, rg, gradient=True)
        assert flops_sep < g.flops(True)        # the separable analysis did run
    finally:
        g.set_analysis("auto")
    for key in sep:
        assert field_err(key, sep[key], dense[key]) <= TOL_FP64, key
    rng = np.random.default_rng(40)
    cells = np.sort(rng.choice(spec.n_ang, 24, replace=False))
    ref = oracle_grid(spec).solve(ry, rg, gradient=True, cells=cells)
    j, k = np.divmod(cells, spec.n_phi)
    for q in ("yin", "yang"):
        assert phi_err(sep["phi_" + q][:, j, k], ref["phi_" + q]) <= TOL_FP64, q
        assert grad_err(sep["grad_" + q][:, :, j, k], ref["grad_" + q]) <= TOL_FP64, q


def test_long_radial_grid_uses_the_chunked_scan(yy, oracle_grid):
    """n_r = 1000 (> 768): the radial sums run as the two-kernel chunked scan
    (per-chunk affine maps, then the composed starts).  Float64 at 1e-13 and
    FP16X2 at its tolerance against the oracle."""
    spec = inputs.GridSpec("long_r", np.logspace(-4, 0, 1001), 16, 48, 0.2, 0.1, 10)
    g = _grid(yy, spec)
    g.prepare("fp16x2")
    ry, rg = inputs.pns_density(spec, 31, 0.05)
    ref = oracle_grid(spec).solve(ry, rg, gradient=True)
    out = gpu_solve(g, ry, rg, gradient=True)
    half = gpu_solve(g, ry, rg, gradient=True, prec="fp16x2")
    for q in ("yin", "yang"):
        assert phi_err(out["phi_" + q], ref["phi_" + q]) <= TOL_FP64, q
        assert grad_err(out["grad_" + q], ref["grad_" + q]) <= TOL_FP64, q
        assert phi_err(half["phi_" + q], ref["phi_" + q]) <= 1e-6, q
        assert grad_err(half["grad_" + q], ref["grad_" + q]) <= 4e-6, q


@pytest.mark.parametrize("lmax", [60, 80])
def test_high_degree(yy, oracle_grid, lmax):
    """l_max = 60 and 80 (the cap) on a small grid: the normalised polar
    tables, the rotation between the patches and the scans at high degree,
    float64 at 1e-13."""
    spec = inputs.GridSpec(f"lmax{lmax}", np.logspace(-2, 0, 9), 40, 120, 0.0, 0.0, lmax)
    g = _grid(yy, spec)
    ry, rg = inputs.pns_density(spec, 32, 0.08)
    out = gpu_solve(g, ry, rg, gradient=True)
    rng = np.random.default_rng(lmax)
    cells = np.sort(rng.choice(spec.n_ang, 40, replace=False))
    ref = oracle_grid(spec).solve(ry, rg, gradient=True, cells=cells)
    j, k = np.divmod(cells, spec.n_phi)
    for q in ("yin", "yang"):
        assert phi_err(out["phi_" + q][:, j, k], ref["phi_" + q]) <= TOL_FP64, q
        assert grad_err(out["grad_" + q][:, :, j, k], ref["grad_" + q]) <= TOL_FP64, q


def test_ragged_small_grid(yy):
    """Odd sizes that leave ragged tiles everywhere (n_r, n_ang, n_lm not
    multiples of any tile), r_edges[0] = 0, unequal buffers."""
    from oracle import OracleGrid
    spec = inputs.GridSpec("ragged", np.concatenate([[0.0], np.logspace(-2, 0, 70)]), 13, 37,
                           0.06, 0.02, 11, 0.5)
    rng = np.random.default_rng(32)
    ry = rng.uniform(0.0, 1.0, (spec.n_r, 13, 37))
    rg = rng.uniform(0.0, 1.0, (spec.n_r, 13, 37))
    g = yy.Grid.from_spec(spec)
    out = gpu_solve(g, ry, rg, gradient=True)
    ref = OracleGrid(spec.r_edges, 13, 37, 0.06, 0.02, 11, 0.5).solve(ry, rg, gradient=True)
    for q in ("yin", "yang"):
        assert phi_err(out["phi_" + q], ref["phi_" + q]) <= TOL_FP64
        assert grad_err(out["grad_" + q], ref["grad_" + q]) <= TOL_FP64
    g.close()


def test_degenerate_lmax0_single_zone(yy):
    """l_max = 0 (monopole only), one radial zone, a 1 x 1 patch."""
    from oracle import OracleGrid
    r = np.array([0.1, 1.0])
    g = yy.Grid(r, 1, 1, 0.0, 0.0, 0, 1.0)
    ry = np.full((1, 1, 1), 2.0)
    rg = np.full((1, 1, 1), 3.0)
    out = gpu_solve(g, ry, rg, gradient=True)
    ref = OracleGrid(r, 1, 1, 0.0, 0.0, 0, 1.0).solve(ry, rg, gradient=True)
    for q in ("yin", "yang"):
        assert phi_err(out["phi_" + q], ref["phi_" + q]) <= TOL_FP64
        assert grad_err(out["grad_" + q][0], ref["grad_" + q][0]) <= TOL_FP64
    g.close()


def test_zero_density_gives_zero(yy):
    spec = inputs.tiny_grid()
    g = _grid(yy, spec)
    z = np.zeros((spec.n_r, spec.n_theta, spec.n_phi))
    out = gpu_solve(g, z, z, gradient=True)
    for v in out.values():
        assert np.all(v == 0.0)


def test_swap_symmetry_bitwise_and_determinism(yy):
    spec = inputs.mid_grid()
    g = _grid(yy, spec)
    ry, rg = inputs.density_for(spec)
    a = gpu_solve(g, ry, rg, gradient=True)
    b = gpu_solve(g, rg, ry, gradient=True)
    c = gpu_solve(g, ry, rg, gradient=True)
    assert np.array_equal(a["phi_yin"], b["phi_yang"])
    assert np.array_equal(a["phi_yang"], b["phi_yin"])
    assert np.array_equal(a["grad_yin"], b["grad_yang"])
    for key in a:
        assert np.array_equal(a[key], c[key])


def test_linearity(yy):
    spec = inputs.tiny_grid()
    g = _grid(yy, spec)
    rng = np.random.default_rng(33)
    shape = (spec.n_r, spec.n_theta, spec.n_phi)
    r1 = [rng.uniform(0, 1, shape) for _ in range(2)]
    r2 = [rng.uniform(0, 1, shape) for _ in range(2)]
    a = gpu_solve(g, *r1)["phi_yin"]
    b = gpu_solve(g, *r2)["phi_yin"]
    c = gpu_solve(g, 2 * r1[0] - 3 * r2[0], 2 * r1[1] - 3 * r2[1])["phi_yin"]
    assert np.abs(c - (2 * a - 3 * b)).max() <= 1e-13 * np.abs(c).max()


def test_host_entry_point_matches_device_path(yy):
    import torch
    spec = inputs.tiny_grid()
    g = _grid(yy, spec)
    ry, rg = inputs.density_for(spec)
    dev = gpu_solve(g, ry, rg, gradient=True)
    shape = (spec.n_r, spec.n_theta, spec.n_phi)
    h = {k: torch.empty(s, dtype=torch.float64).pin_memory()
         for k, s in (("py", shape), ("pg", shape), ("gy", (3,) + shape), ("gg", (3,) + shape))}
    ryt = torch.from_numpy(np.ascontiguousarray(ry)).pin_memory()
    rgt = torch.from_numpy(np.ascontiguousarray(rg)).pin_memory()
    st = yy.yy_potential_host(g.handle, ryt, rgt, h["py"], h["pg"], h["gy"], h["gg"], yy.YY_FP64,
                              torch.cuda.current_stream())
    assert st == yy.YY_OK
    assert np.array_equal(h["py"].numpy(), dev["phi_yin"])
    assert np.array_equal(h["gg"].numpy(), dev["grad_yang"])


def test_pipelined_host_calls_match_device_path(yy):
    """yy_potential_host_async: five calls in a row with different densities
    and their own host buffers (the staging sets alternate and the copies
    overlap); after yy_potential_host_wait each result equals the device
    path bitwise, in float64 and in FP16X2."""
    import torch
    spec = inputs.mid_grid()
    g = _grid(yy, spec)
    g.prepare("fp16x2")
    ry, rg = inputs.density_for(spec)
    shape = (spec.n_r, spec.n_theta, spec.n_phi)
    stream = torch.cuda.current_stream()
    for prec in ("fp64", "fp16x2"):
        calls = []
        for i in range(5):
            f = 1.0 + 0.25 * i
            rin = [torch.from_numpy(np.ascontiguousarray(a * f)).pin_memory() for a in (ry, rg)]
            out = [torch.empty(shape, dtype=torch.float64).pin_memory() for _ in range(2)] + \
                  [torch.empty((3,) + shape, dtype=torch.float64).pin_memory() for _ in range(2)]
            st = yy.yy_potential_host_async(g.handle, rin[0], rin[1], out[0], out[1], out[2], out[3],
                                            yy.PRECISIONS[prec], stream)
            assert st == yy.YY_OK
            calls.append((f, rin, out))
        assert yy.yy_potential_host_wait(g.handle) == yy.YY_OK
        for f, rin, out in calls:
            ref = gpu_solve(g, ry * f, rg * f, gradient=True, prec=prec)
            for key, o in zip(("phi_yin", "phi_yang", "grad_yin", "grad_yang"), out):
                assert np.array_equal(o.numpy(), ref[key]), (prec, f, key)


def test_error_paths(yy):
    import torch
    spec = inputs.tiny_grid()
    g = _grid(yy, spec)
    x = torch.zeros((spec.n_r, spec.n_theta, spec.n_phi), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    # one gradient pointer only
    assert yy.yy_potential(g.handle, x, x, y, y, y, None) == yy.YY_ERR_INVALID_ARG
    # misaligned pointer
    assert yy.yy_potential(g.handle, x.data_ptr() + 8, x, y, y) == yy.YY_ERR_INVALID_ARG
    # unknown precision
    assert yy.yy_potential(g.handle, x, x, y, y, prec=9) == yy.YY_ERR_INVALID_ARG
    assert yy.yy_last_device_status(g.handle) == yy.YY_OK


def test_allocation_failure_is_reported_cleanly(yy):
    spec = inputs.tiny_grid()
    for n in (0, 3, 7):
        yy.yy_debug_fail_alloc_after(n)
        st, h = yy.yy_grid_create(spec.r_edges, spec.n_theta, spec.n_phi, spec.delta_theta,
                                  spec.delta_phi, spec.lmax)
        yy.yy_debug_fail_alloc_after(-1)
        assert st == yy.YY_ERR_OOM and not h
    # the library still works afterwards
    g = yy.Grid.from_spec(spec)
    g.close()


@pytest.mark.parametrize("analysis", ["auto", "dense"])
def test_fp32_path_tolerance(yy, oracle_grid, analysis):
    """float32 on CUDA cores (float64 tables cast once, float64 scans).
    Default (separable stages, sums of short chains with the monopole added
    last): Phi <= 1e-6 pointwise, -grad Phi <= 1e-6 normwise (worst measured
    2.1e-7 and 1.9e-7).  Dense contractions, long fp32 chains: 1e-5 and 1e-5
    (worst measured 2.4e-6 and 1.9e-6)."""
    spec = inputs.mid_grid()
    g = _grid(yy, spec)
    g.prepare("fp32")
    ry, rg = inputs.density_for(spec)
    g.set_analysis(analysis)
    try:
        out = gpu_solve(g, ry, rg, gradient=True, prec="fp32")
    finally:
        g.set_analysis("auto")
    ref = oracle_grid(spec).solve(ry, rg, gradient=True)
    tol_phi, tol_g = (1e-6, 1e-6) if analysis == "auto" else (1e-5, 1e-5)
    for q in ("yin", "yang"):
        assert phi_err(out["phi_" + q], ref["phi_" + q]) <= tol_phi
        assert grad_err(out["grad_" + q], ref["grad_" + q]) <= tol_g
