"""Tensor-core forms (tcgen05) against the float64 oracle.

Stated tolerances (Phi: the largest pointwise relative error |dPhi|/|Phi|;
-grad Phi: normwise, max |dg| / max |g|), over the whole field:
  FP16X2, BF16X3  Phi <= 1e-6 (the target; worst measured 5.3e-7, tiny grid)
                  -grad Phi <= 4e-6 (4x the worst measured, 8.8e-7)
  TF32            Phi <= 5e-4, -grad Phi <= 7e-4 (about 5x and 4.5x the worst
                  measured, 1.0e-4 and 1.5e-4; TF32 misses the 1e-6 target)
The split forms keep about 22 (fp16 x 2) or 24 (bf16 x 3) significant bits
per operand; the bound comes from the fp32 accumulation in tensor memory
(about 2^-24 per accumulation step, a few hundred steps per output) with the
monopole done in float64.  The gradient weights mode l by about l relative
to Phi, so its bound is larger.  TF32 keeps 11 bits.
"""

import numpy as np
import pytest

from paper_1806_04593_gb300 import inputs

from .gpu_common import gpu_solve, grad_err, lib, phi_err, require_gpu

pytestmark = pytest.mark.gpu

TOL = {"fp16x2": (1e-6, 4e-6), "bf16x3": (1e-6, 4e-6), "tf32": (5e-4, 7e-4)}


@pytest.fixture(scope="module")
def yy():
    require_gpu()
    return lib()


_GRIDS = {}


def _grid(yy, spec):
    if spec.name not in _GRIDS:
        _GRIDS[spec.name] = yy.Grid.from_spec(spec)
    return _GRIDS[spec.name]


@pytest.mark.parametrize("analysis", ["auto", "separable", "dense"])
@pytest.mark.parametrize("prec", ["fp16x2", "bf16x3", "tf32"])
@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_tensor_form_matches_oracle(yy, oracle_grid, prec, name, analysis):
    """Both analysis evaluations: the separable one (fp32 azimuthal stage,
    float64 m = 0 sums) and the dense tensor-core contraction."""
    spec = inputs.GRIDS[name]()
    g = _grid(yy, spec)
    g.prepare(prec)
    ry, rg = inputs.density_for(spec)
    g.set_analysis(analysis)
    try:
        out = gpu_solve(g, ry, rg, gradient=True, prec=prec)
    finally:
        g.set_analysis("auto")
    assert yy.yy_last_device_status(g.handle) == yy.YY_OK
    ref = oracle_grid(spec).solve(ry, rg, gradient=True)
    tol_phi, tol_g = TOL[prec]
    for q in ("yin", "yang"):
        assert phi_err(out["phi_" + q], ref["phi_" + q]) <= tol_phi, (q, prec)
        assert grad_err(out["grad_" + q], ref["grad_" + q]) <= tol_g, (q, prec)


@pytest.mark.parametrize("analysis", ["auto", "separable", "dense"])
@pytest.mark.parametrize("prec", ["fp16x2", "bf16x3"])
def test_tensor_form_production_sampled(yy, oracle_grid, prec, analysis):
    spec = inputs.production_grid()
    g = _grid(yy, spec)
    g.prepare(prec)
    ry, rg = inputs.density_for(spec)
    g.set_analysis(analysis)
    try:
        out = gpu_solve(g, ry, rg, gradient=True, prec=prec)
    finally:
        g.set_analysis("auto")
    assert yy.yy_last_device_status(g.handle) == yy.YY_OK
    rng = np.random.default_rng(41)
    cells = np.sort(rng.choice(spec.n_ang, 64, replace=False))
    ref = oracle_grid(spec).solve(ry, rg, gradient=True, cells=cells)
    j, k = np.divmod(cells, spec.n_phi)
    tol_phi, tol_g = TOL[prec]
    for q in ("yin", "yang"):
        assert phi_err(out["phi_" + q][:, j, k], ref["phi_" + q]) <= tol_phi
        assert grad_err(out["grad_" + q][:, :, j, k], ref["grad_" + q]) <= tol_g


def test_tensor_form_ragged_sizes(yy):
    """Sizes that are multiples of no tile: partial M, N and K tiles."""
    from oracle import OracleGrid
    spec = inputs.GridSpec("ragged_tc", np.logspace(-2, 0, 131), 17, 41, 0.03, 0.05, 13, 1.0)
    rng = np.random.default_rng(42)
    ry = rng.uniform(0.5, 1.5, (spec.n_r, 17, 41))
    rg = rng.uniform(0.5, 1.5, (spec.n_r, 17, 41))
    g = yy.Grid.from_spec(spec)
    ref = OracleGrid(spec.r_edges, 17, 41, 0.03, 0.05, 13).solve(ry, rg, gradient=True)
    for prec in ("fp16x2", "bf16x3", "tf32"):
        g.prepare(prec)
        out = gpu_solve(g, ry, rg, gradient=True, prec=prec)
        tol_phi, tol_g = TOL[prec]
        for q in ("yin", "yang"):
            assert phi_err(out["phi_" + q], ref["phi_" + q]) <= tol_phi, prec
            assert grad_err(out["grad_" + q], ref["grad_" + q]) <= tol_g, prec
    assert yy.yy_last_device_status(g.handle) == yy.YY_OK
    g.close()


def test_tensor_form_deterministic_and_swap_symmetric(yy):
    spec = inputs.mid_grid()
    g = _grid(yy, spec)
    g.prepare("fp16x2")
    ry, rg = inputs.density_for(spec)
    a = gpu_solve(g, ry, rg, gradient=True, prec="fp16x2")
    b = gpu_solve(g, ry, rg, gradient=True, prec="fp16x2")
    c = gpu_solve(g, rg, ry, gradient=True, prec="fp16x2")
    for key in a:
        assert np.array_equal(a[key], b[key]), key
    assert np.array_equal(a["phi_yin"], c["phi_yang"])
    assert np.array_equal(a["grad_yang"], c["grad_yin"])


def test_zero_density_tensor_form(yy):
    spec = inputs.tiny_grid()
    g = _grid(yy, spec)
    g.prepare("fp16x2")
    z = np.zeros((spec.n_r, spec.n_theta, spec.n_phi))
    out = gpu_solve(g, z, z, gradient=True, prec="fp16x2")
    for v in out.values():
        assert np.all(v == 0.0)


def test_unprepared_precision_is_not_supported(yy):
    import torch
    spec = inputs.tiny_grid()
    g = yy.Grid.from_spec(spec)
    x = torch.zeros((spec.n_r, spec.n_theta, spec.n_phi), dtype=torch.float64, device="cuda")
    assert yy.yy_potential(g.handle, x, x, x.clone(), x.clone(), prec=yy.YY_BF16X3) == yy.YY_ERR_NOT_SUPPORTED
    g.close()


def test_separable_tables_built_on_selection(yy):
    """The separable tensor-core tables cost device memory only while the
    separable evaluation is selected, and selecting it before or after the
    form is prepared gives bitwise the same solve."""
    import torch
    spec = inputs.GRIDS["mid"]()
    ry, rg = inputs.density_for(spec)
    a = yy.Grid.from_spec(spec)
    b = yy.Grid.from_spec(spec)
    try:
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        a.prepare("fp16x2")                        # AUTO: dense, no separable tables
        free1 = torch.cuda.mem_get_info()[0]
        a.set_analysis("separable")                # builds them now
        free2 = torch.cuda.mem_get_info()[0]
        assert free2 < free1 <= free0
        b.set_analysis("separable")
        b.prepare("fp16x2")                        # builds them while preparing
        out_a = gpu_solve(a, ry, rg, gradient=True, prec="fp16x2")
        out_b = gpu_solve(b, ry, rg, gradient=True, prec="fp16x2")
        for key in out_a:
            assert np.array_equal(out_a[key], out_b[key]), key
        assert yy.yy_last_device_status(a.handle) == yy.YY_OK
    finally:
        a.close()
        b.close()


def test_long_rows_streaming_packing(yy):
    """Density rows of 2 760 cells (even, longer than a warp's share) go
    through the streaming packing: 194 rows over at most one block per SM,
    so blocks walk several rows.  Against the oracle for every form; a
    density pointer off the 16-byte grid is refused."""
    import torch

    from oracle import OracleGrid
    spec = inputs.GridSpec("long_rows_tc", np.logspace(-2, 0, 98), 30, 92, 0.02, 0.04, 12, 1.0)
    rng = np.random.default_rng(43)
    ry = rng.uniform(0.5, 1.5, (spec.n_r, 30, 92))
    rg = rng.uniform(0.5, 1.5, (spec.n_r, 30, 92))
    ref = OracleGrid(spec.r_edges, 30, 92, 0.02, 0.04, 12).solve(ry, rg, gradient=True)
    g = yy.Grid.from_spec(spec)
    try:
        for prec in ("fp16x2", "bf16x3", "tf32"):
            g.prepare(prec)
            out = gpu_solve(g, ry, rg, gradient=True, prec=prec)
            tol_phi, tol_g = TOL[prec]
            for q in ("yin", "yang"):
                assert phi_err(out["phi_" + q], ref["phi_" + q]) <= tol_phi, prec
                assert grad_err(out["grad_" + q], ref["grad_" + q]) <= tol_g, prec
        assert yy.yy_last_device_status(g.handle) == yy.YY_OK
        buf = torch.zeros(ry.size + 1, dtype=torch.float64, device="cuda")
        off = buf[1:].view(ry.shape)
        phi = torch.empty_like(off)
        assert yy.yy_potential(g.handle, off, off, phi, phi.clone(), prec=yy.YY_FP16X2) == yy.YY_ERR_INVALID_ARG
    finally:
        g.close()
