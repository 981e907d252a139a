"""yy_radial_scan_static: the allocation-free scan entry point.

It serves callers that cannot allocate device memory where they need the
radial sums: applications whose device memory belongs to their own pool,
plugin hosts that forbid the allocator, loops where cudaMalloc may not run.
Its output is checked against the oracle's radial sums (Eqs. phiin/phiout at
the interfaces r_n^+, computed there by direct powers and cumulative sums) and
against the coefficients the regular solve produces from the same moments,
on consecutive calls that reuse the shared static scratch.  This file is
collected last so that a failure here never hides the other tests.
"""

import math

import numpy as np
import pytest

from paper_1806_04593_gb300 import inputs

from .gpu_common import K_lm, lib, mode_index, require_gpu

pytestmark = pytest.mark.gpu

SCRATCH_DOUBLES = 1 << 21


def _oracle_coefficients(r_edges, lmax, G, A_C, A_S):
    """The library's moment layout and expected coefficients from the
    oracle's radial sums: moments idx(l, m) = K_lm A, and
    Q = -G 4 pi / (2l+1) K_lm U, Q_r = G 4 pi / (2l+1) K_lm dU, Q_t = -Q / r."""
    from oracle import OracleGrid
    from oracle.yinyang import normalisation, radial_integrals
    og = OracleGrid.__new__(OracleGrid)          # only the radial-sum terms are needed
    og.r_edges = np.asarray(r_edges, dtype=np.float64)
    og.n_r = og.r_edges.size - 1
    og.lmax = lmax
    og.R_in, og.R_out = radial_integrals(lmax, og.r_edges)
    K = K_lm(normalisation(lmax))
    modes = mode_index(lmax)
    n_r = og.n_r
    mom = np.zeros((2, n_r, len(modes)))
    exp = np.zeros((3, 2, n_r, len(modes)))
    r = og.r_edges[1:]
    for p in range(2):
        u = og.radial_sums(A_C[p], A_S[p])
        for idx, (l, m, kind) in enumerate(modes):
            src = A_C[p] if kind == "c" else A_S[p]
            mom[p, :, idx] = K[l, m] * src[:, l, m]
            U = u["U_C" if kind == "c" else "U_S"][:, l, m]
            dU = u["dU_C" if kind == "c" else "dU_S"][:, l, m]
            f = G * 4 * math.pi / (2 * l + 1) * K[l, m]
            exp[0, p, :, idx] = -f * U
            exp[1, p, :, idx] = f * dU
            exp[2, p, :, idx] = f * U / r
    return mom.reshape(2 * n_r, -1), exp.reshape(3, 2 * n_r, -1)


def _blockwise_error(got, exp, lmax):
    """Largest error per (coefficient set, patch, degree l) block, relative to
    the block's largest value: the degrees span many orders of magnitude."""
    n_rows = got.shape[1] // 2
    worst = 0.0
    for c in range(3):
        for p in range(2):
            rows = slice(p * n_rows, (p + 1) * n_rows)
            for l in range(lmax + 1):
                cols = slice(l * l, (l + 1) * (l + 1))
                ref = exp[c, rows, cols]
                scale = np.abs(ref).max()
                if scale == 0.0:
                    assert np.all(got[c, rows, cols] == 0.0)
                    continue
                worst = max(worst, float(np.abs(got[c, rows, cols] - ref).max() / scale))
    return worst


def _static_scan(yy, r_edges, n_r, lmax, G, moments, calls=2):
    import torch
    dev = torch.device("cuda", 0)
    r_dev = torch.from_numpy(np.ascontiguousarray(r_edges, dtype=np.float64)).to(dev)
    m_dev = torch.from_numpy(np.ascontiguousarray(moments, dtype=np.float64)).to(dev)
    outs = []
    for _ in range(calls):
        coeff = torch.full((3, 2 * n_r, (lmax + 1) ** 2), float("nan"), dtype=torch.float64, device=dev)
        st = yy.yy_radial_scan_static(r_dev, n_r, lmax, G, m_dev, coeff, torch.cuda.current_stream())
        assert st == yy.YY_OK, yy.yy_status_string(st)
        torch.cuda.synchronize()
        outs.append(coeff.cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    assert np.all(np.isfinite(outs[0]))
    return outs[0]


def test_static_scan_matches_oracle_and_solve_twice():
    """Mid grid (200 zones, l_max = 15): the oracle's moments of the seeded
    density through the static scan agree with the oracle's radial sums, and
    the solve's own combined moments agree with the solve's coefficients."""
    import torch
    from oracle import OracleGrid
    require_gpu()
    yy = lib()
    spec = inputs.mid_grid()
    ry, rg = inputs.density_for(spec)
    og = OracleGrid(spec.r_edges, spec.n_theta, spec.n_phi, spec.delta_theta, spec.delta_phi, spec.lmax, spec.G)
    (cy, sy), (cg, sg) = og.analysis(ry), og.analysis(rg)
    mom, exp = _oracle_coefficients(spec.r_edges, spec.lmax, spec.G, (cy, cg), (sy, sg))
    got = _static_scan(yy, spec.r_edges, spec.n_r, spec.lmax, spec.G, mom)
    assert _blockwise_error(got, exp, spec.lmax) <= 1e-12

    grid = yy.Grid.from_spec(spec)
    dev = torch.device("cuda", 0)
    grid.solve(torch.from_numpy(ry).to(dev), torch.from_numpy(rg).to(dev))
    torch.cuda.synchronize()
    moments = grid.table(yy.YY_TABLE_MOMENTS_TOTAL)    # the regular entry point's scan input
    expected = grid.table(yy.YY_TABLE_COEFF).reshape(3, 2 * spec.n_r, -1)
    got = _static_scan(yy, spec.r_edges, spec.n_r, spec.lmax, spec.G, moments)
    assert _blockwise_error(got, expected, spec.lmax) <= 1e-13
    grid.close()


@pytest.mark.parametrize("case", ["long", "from_zero", "at_limit", "lmax80", "many_zones"])
def test_static_scan_edge_cases_against_oracle(case):
    """Random moments through the static scan against the oracle's radial
    sums: 1000 zones (32 radii per lane), a grid whose first zone starts at
    r = 0 (empty-ball base case, outer factor of zone 0 unused), the largest
    accepted size 2 n_r (l_max+1)^2 = 2^21 exactly, l_max = 80, and 8000
    zones (more than the shared-memory factor table holds: the kernel that
    computes the factors per warp)."""
    require_gpu()
    yy = lib()
    n_r, lmax, r = {
        "long": (1000, 15, np.logspace(-3, 0, 1001)),
        "from_zero": (64, 12, np.concatenate([[0.0], np.logspace(-3, 0, 64)])),
        "at_limit": (1024, 31, np.logspace(-3, 0, 1025)),
        "lmax80": (100, 80, np.logspace(-1.5, 0, 101)),
        "many_zones": (8000, 3, np.logspace(-3, 0, 8001)),
    }[case]
    assert 2 * n_r * (lmax + 1) ** 2 <= SCRATCH_DOUBLES
    rng = np.random.default_rng(77)
    A_C = rng.standard_normal((2, n_r, lmax + 1, lmax + 1))
    A_S = rng.standard_normal((2, n_r, lmax + 1, lmax + 1))
    A_S[..., 0] = 0.0                                  # no sine term at m = 0
    mom, exp = _oracle_coefficients(r, lmax, 1.0, A_C, A_S)
    got = _static_scan(yy, r, n_r, lmax, 1.0, mom)
    assert _blockwise_error(got, exp, lmax) <= 1e-12, case


def test_static_scan_rejects_sizes_beyond_the_scratch():
    import torch
    require_gpu()
    yy = lib()
    dev = torch.device("cuda", 0)
    r = torch.from_numpy(np.logspace(-3, 0, 1026)).to(dev)
    m = torch.zeros((2 * 1025, 32 * 32), dtype=torch.float64, device=dev)
    q = torch.zeros((3, 2 * 1025, 32 * 32), dtype=torch.float64, device=dev)
    # one zone more than the largest accepted size at l_max = 31
    assert yy.yy_radial_scan_static(r, 1025, 31, 1.0, m, q, None) == yy.YY_ERR_INVALID_ARG
    assert yy.yy_radial_scan_static(r, 10, 81, 1.0, m, q, None) == yy.YY_ERR_INVALID_ARG
    assert torch.count_nonzero(q).item() == 0          # nothing was launched
