"""Homogeneous-ellipsoid validation (§5) on the GPU path, low resolution.

The ellipsoid (a = 0.5, b = 1.5 a, c = 2 a, unit density, turned by pi/8
about z) on the §5 "LR" grids: 400 equidistant zones on [0, c] with 2-degree
cells, as a Yin-Yang grid and as a full spherical polar grid.  The reference
is the semi-analytic potential (Carlson integrals) at the output points.
Expected, as §5 reports: the maximum relative error falls as l_max grows,
both grids give nearly the same error, and (here) the reduced-precision form
is indistinguishable from float64 at this accuracy.  The bounds come from the
measured sweep (tests/ellipsoid_sweep.py): 1.88e-2 at l_max = 5 and
2.8e-4 / 3.2e-4 (Yin-Yang / polar) at l_max = 40.
"""

import numpy as np
import pytest

from .gpu_common import lib, require_gpu

pytestmark = pytest.mark.gpu

LMAX = (5, 10, 20, 40)


@pytest.fixture(scope="module")
def yy():
    require_gpu()
    return lib()


@pytest.fixture(scope="module")
def sweep(yy):
    from . import ellipsoid_sweep as es
    out = {}
    for kind, spec in es.grid_specs("LR").items():
        rho, ref = es.reference(spec)
        errs = {L: es.errors(es.solve(spec, L, rho, "fp64"), ref) for L in LMAX}
        errs["fp16x2"] = es.errors(es.solve(spec, LMAX[-1], rho, "fp16x2"), ref)
        out[kind] = errs
    return out


@pytest.mark.parametrize("kind", ["yinyang", "polar"])
def test_error_falls_with_lmax(sweep, kind):
    e = [sweep[kind][L][0] for L in LMAX]
    assert all(b < a for a, b in zip(e, e[1:])), e
    assert 0.01 <= e[0] <= 0.03          # truncation at l_max = 5 (measured 1.88e-2)
    assert e[-1] <= 5e-4                 # measured 2.8e-4 (Yin-Yang), 3.2e-4 (polar)


def test_yinyang_and_polar_agree(sweep):
    for L in LMAX:
        a, b = sweep["yinyang"][L][0], sweep["polar"][L][0]
        assert max(a, b) / min(a, b) <= 1.5, (L, a, b)


@pytest.mark.parametrize("kind", ["yinyang", "polar"])
def test_fp16x2_matches_fp64_at_this_accuracy(sweep, kind):
    e64, e16 = sweep[kind][LMAX[-1]][0], sweep[kind]["fp16x2"][0]
    assert abs(e16 - e64) <= 0.01 * e64
