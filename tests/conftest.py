import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built library")


_GRID_CACHE = {}


@pytest.fixture(scope="session")
def oracle_grid():
    """Session-cached oracle grids by spec name."""
    from oracle import OracleGrid, OraclePolarGrid

    def get(spec):
        polar = bool(getattr(spec, "polar", False))
        key = (spec.name, polar, spec.n_r, spec.n_theta, spec.n_phi, spec.lmax,
               spec.delta_theta, spec.delta_phi, float(spec.r_edges[0]), float(spec.r_edges[-1]))
        if key not in _GRID_CACHE:
            if polar:
                _GRID_CACHE[key] = OraclePolarGrid(spec.r_edges, spec.n_theta, spec.n_phi, spec.lmax, spec.G)
            else:
                _GRID_CACHE[key] = OracleGrid(spec.r_edges, spec.n_theta, spec.n_phi,
                                              spec.delta_theta, spec.delta_phi, spec.lmax, spec.G)
        return _GRID_CACHE[key]

    return get
