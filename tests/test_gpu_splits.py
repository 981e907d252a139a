"""The dense analysis gives the same moments for every K split.

Sec. 3 (the paragraph on the global summation of A_C and A_S): the order in
which the partial sums of the moments are added changed A by rounding, and
the paper made A reproducible with double-double sums.  Here the K axis of
the dense analysis (the n_ang cells) is cut into segments fixed by the grid's
sizes; each segment is summed in one fixed order into a partial of its own,
a split takes whole segments, and the partials are added in segment order.
So the split -- which the batch tuner picks per field for speed -- leaves the
moments and everything computed from them bitwise unchanged.  Checked on the
1-degree grid (K = 24300: 95 accumulator fills of the tensor-core forms) for
the three tensor-core forms and for the float64 CUDA-core contraction (also
the analysis of YY_FP64_OZAKI with the dense evaluation), from one tile
along K up to the default (which is also the largest: one segment per tile).
"""

import numpy as np
import pytest

from paper_1806_04593_gb300 import inputs

from .gpu_common import gpu_solve, lib, phi_err, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def production():
    require_gpu()
    yy = lib()
    spec = inputs.production_grid()
    ry, rg = inputs.density_for(spec)
    grid = yy.Grid.from_spec(spec)
    grid.set_analysis("dense")
    yield yy, spec, grid, ry, rg
    grid.close()


def _splits_to_try(grid, prec):
    cur, rule, cap = grid.analysis_splits(prec)
    assert cur == rule and 1 <= rule <= cap
    return sorted({1, 2, 3, rule // 2, rule - 1, rule, cap} & set(range(1, cap + 1))), rule, cap


@pytest.mark.parametrize("prec", ["fp16x2", "bf16x3", "tf32", "fp64", "fp64_ozaki"])
def test_moments_and_phi_do_not_depend_on_the_split(production, prec):
    yy, spec, grid, ry, rg = production
    if prec != "fp64":
        grid.prepare(prec)
    tried, rule, cap = _splits_to_try(grid, prec)
    assert cap >= 4, (prec, rule, cap)     # several segments, so the splits really differ
    ref = None
    effective = set()
    for s in tried:
        grid.set_analysis_splits(prec, s)
        cur, _, _ = grid.analysis_splits(prec)
        assert 1 <= cur <= s
        effective.add(cur)
        out = gpu_solve(grid, ry, rg, gradient=True, prec=prec)
        A = grid.table(yy.YY_TABLE_MOMENTS).copy()
        if ref is None:
            ref = (A, out)
            continue
        assert np.array_equal(A, ref[0]), (prec, s)
        for key in out:
            assert np.array_equal(out[key], ref[1][key]), (prec, s, key)
    assert len(effective) >= 4, effective
    grid.set_analysis_splits(prec, 0)
    assert grid.analysis_splits(prec)[0] == rule


def test_split_bounds_are_checked(production):
    yy, spec, grid, ry, rg = production
    grid.prepare("fp16x2")
    for prec in ("fp16x2", "fp64"):
        cur, rule, cap = grid.analysis_splits(prec)
        with pytest.raises(yy.YYError):
            grid.set_analysis_splits(prec, cap + 1)
        with pytest.raises(yy.YYError):
            grid.set_analysis_splits(prec, -1)
        assert grid.analysis_splits(prec)[0] == cur


def test_split_solve_still_matches_the_float64_path(production):
    """The segment partials change where the sums are cut, not what they
    add up to: the finest split of FP16X2 stays within the form's Phi
    tolerance (1e-6 pointwise) of the float64 result."""
    yy, spec, grid, ry, rg = production
    grid.prepare("fp16x2")
    ref = gpu_solve(grid, ry, rg, prec="fp64")
    cap = grid.analysis_splits("fp16x2")[2]
    grid.set_analysis_splits("fp16x2", cap)
    got = gpu_solve(grid, ry, rg, prec="fp16x2")
    grid.set_analysis_splits("fp16x2", 0)
    assert phi_err(got["phi_yin"], ref["phi_yin"]) <= 1e-6
    assert phi_err(got["phi_yang"], ref["phi_yang"]) <= 1e-6
