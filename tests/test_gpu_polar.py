"""The full spherical polar grid of §2 (yy_polar_grid_create) against the
float64 oracle's polar grid: float64 at 1e-13 (the 1e-12 bar with room
for regressions to show) with both analysis evaluations, the tensor-core
forms at their stated tolerances (Phi pointwise 1e-6 and -grad Phi normwise
4e-6 for FP16X2 / BF16X3, 5e-4 / 7e-4 for TF32), a 1-degree grid on sampled
cells, and the one-patch argument rules.
"""

import numpy as np
import pytest

from paper_1806_04593_gb300 import inputs

from .gpu_common import grad_err, lib, phi_err, require_gpu

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-13
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


def _solve(g, rho, prec="fp64"):
    import torch
    r = torch.as_tensor(np.ascontiguousarray(rho), device=torch.device("cuda", 0))
    out = g.solve(r, gradient=True, prec=prec)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("analysis", ["separable", "dense"])
@pytest.mark.parametrize("name", ["tiny_polar", "mid_polar"])
def test_polar_fp64_matches_oracle(yy, oracle_grid, name, analysis):
    spec = inputs.GRIDS[name]()
    g = _grid(yy, spec)
    rho, none = inputs.pns_density(spec, 3, 0.05) if name == "mid_polar" else inputs.tiny_density(spec)
    assert none is None
    g.set_analysis(analysis)
    try:
        out = _solve(g, rho)
    finally:
        g.set_analysis("auto")
    assert yy.yy_last_device_status(g.handle) == yy.YY_OK
    ref = oracle_grid(spec).solve(rho, gradient=True)
    assert phi_err(out["phi"], ref["phi"]) <= TOL_FP64
    assert grad_err(out["grad"], ref["grad"]) <= TOL_FP64


@pytest.mark.parametrize("prec", ["fp16x2", "bf16x3", "tf32"])
def test_polar_tensor_forms_match_oracle(yy, oracle_grid, prec):
    spec = inputs.mid_polar_grid()
    g = _grid(yy, spec)
    g.prepare(prec)
    rho, _ = inputs.pns_density(spec, 3, 0.05)
    out = _solve(g, rho, prec)
    assert yy.yy_last_device_status(g.handle) == yy.YY_OK
    ref = oracle_grid(spec).solve(rho, gradient=True)
    tol_phi, tol_g = TOL[prec]
    assert phi_err(out["phi"], ref["phi"]) <= tol_phi
    assert grad_err(out["grad"], ref["grad"]) <= tol_g


def test_polar_one_degree_sampled_cells(yy, oracle_grid):
    """1-degree polar grid (180 x 360), 300 zones, l_max = 25: float64 and
    FP16X2 at every radius on sampled cells."""
    spec = inputs.polar_grid(np.logspace(-4, 0, 301), 180, 360, 25, "one_degree_polar")
    g = _grid(yy, spec)
    g.prepare("fp16x2")
    rho, _ = inputs.pns_density(spec, 4, 0.05)
    out64 = _solve(g, rho)
    out16 = _solve(g, rho, "fp16x2")
    rng = np.random.default_rng(25)
    cells = np.sort(rng.choice(spec.n_ang, 32, replace=False))
    ref = oracle_grid(spec).solve(rho, gradient=True, cells=cells)
    j, k = np.divmod(cells, spec.n_phi)
    assert phi_err(out64["phi"][:, j, k], ref["phi"]) <= TOL_FP64
    assert grad_err(out64["grad"][:, :, j, k], ref["grad"]) <= TOL_FP64
    assert phi_err(out16["phi"][:, j, k], ref["phi"]) <= TOL["fp16x2"][0]
    assert grad_err(out16["grad"][:, :, j, k], ref["grad"]) <= TOL["fp16x2"][1]


def test_polar_argument_rules_and_host_entry(yy):
    import torch
    spec = inputs.tiny_polar_grid()
    g = _grid(yy, spec)
    dev = torch.device("cuda", 0)
    rho, _ = inputs.tiny_density(spec)
    r = torch.as_tensor(rho, device=dev)
    phi = torch.empty_like(r)
    other = torch.empty_like(r)
    # a second patch is refused
    assert yy.yy_potential(g.handle, r, r, phi, other) == yy.YY_ERR_INVALID_ARG
    assert yy.yy_potential(g.handle, r, None, phi, other) == yy.YY_ERR_INVALID_ARG
    st, _ = yy.yy_grid_copy_table(g.handle, yy.YY_TABLE_ROTATION)
    assert st == yy.YY_ERR_NOT_SUPPORTED
    w = g.table(yy.YY_TABLE_WEIGHTS)
    assert np.all(w == 1.0)
    # host-buffer entry point equals the device path bitwise
    dev_out = g.solve(r, gradient=True)
    torch.cuda.synchronize()
    h_phi = np.empty_like(rho)
    h_grad = np.empty((3,) + rho.shape)
    st = yy.yy_potential_host(g.handle, np.ascontiguousarray(rho), None, h_phi, None, h_grad, None)
    assert st == yy.YY_OK
    assert np.array_equal(h_phi, dev_out["phi"].cpu().numpy())
    assert np.array_equal(h_grad, dev_out["grad"].cpu().numpy())
