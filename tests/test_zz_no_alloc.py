"""yy_radial_scan_static: the allocation-free scan entry point.

It is meant for callers that cannot allocate device memory where they need
the radial sums (inside a CUDA graph capture, under an application-owned
memory pool, in loops that must not allocate).  Its output must equal the
coefficients the regular solve produces from the same moments, on
consecutive calls that reuse the shared static scratch.  This file is
collected last so that a failure here never hides the other tests.
"""

import numpy as np
import pytest

from paper_1806_04593_gb300 import inputs

from .gpu_common import lib, require_gpu

pytestmark = pytest.mark.gpu


def test_static_scan_matches_solve_coefficients_twice():
    import torch
    require_gpu()
    yy = lib()
    spec = inputs.mid_grid()
    grid = yy.Grid.from_spec(spec)
    dev = torch.device("cuda", 0)
    ry, rg = inputs.density_for(spec)
    grid.solve(torch.from_numpy(ry).to(dev), torch.from_numpy(rg).to(dev))
    torch.cuda.synchronize()
    moments = grid.table(yy.YY_TABLE_MOMENTS_TOTAL)    # existing entry point's scan input
    expected = grid.table(yy.YY_TABLE_COEFF)           # existing entry point's scan output
    n_lm = grid.n_lm
    r_dev = torch.from_numpy(np.ascontiguousarray(spec.r_edges)).to(dev)
    m_dev = torch.from_numpy(moments).to(dev)
    outs = []
    for _ in range(2):
        coeff = torch.full((3, 2 * spec.n_r, n_lm), float("nan"), dtype=torch.float64, device=dev)
        st = yy.yy_radial_scan_static(r_dev, spec.n_r, spec.lmax, spec.G, m_dev, coeff,
                                      torch.cuda.current_stream())
        assert st == yy.YY_OK, yy.yy_status_string(st)
        torch.cuda.synchronize()
        got = coeff.cpu().numpy().reshape(-1)
        err = np.abs(got - expected).max() / np.abs(expected).max()
        assert err <= 1e-12, err
        outs.append(coeff.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    assert np.all(np.isfinite(outs[0]))
    # sizes beyond the static scratch are rejected before any launch
    big = yy.yy_radial_scan_static(r_dev, 4000, 40, 1.0, m_dev, coeff, None)
    assert big == yy.YY_ERR_INVALID_ARG
    grid.close()
