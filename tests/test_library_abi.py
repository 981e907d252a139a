"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
and exports every function that include/*.h declares."""

import ctypes
import os
import re

import pytest

from paper_1806_04593_gb300 import build as yybuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(yy_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    return yybuild.build()


def test_headers_declare_the_boundary():
    names = _declared_functions()
    for required in ("yy_grid_create", "yy_polar_grid_create", "yy_potential", "yy_destroy", "yy_potential_host",
                     "yy_grid_prepare", "yy_last_device_status", "yy_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in sorted(_declared_functions()):
        assert hasattr(lib, name), name


def test_status_strings_without_gpu(lib_path):
    from paper_1806_04593_gb300 import yy
    assert yy.yy_status_string(yy.YY_OK) == "ok"
    assert "invalid" in yy.yy_status_string(yy.YY_ERR_INVALID_ARG)
    assert yy.yy_status_string(99) == "unknown status"


def test_invalid_arguments_rejected_on_host(lib_path):
    """Argument checks run before any CUDA call, so they work without a GPU."""
    import numpy as np
    from paper_1806_04593_gb300 import yy
    r = np.logspace(-3, 0, 9)
    bad = [
        (r[::-1], 4, 12, 0.0, 0.0, 4),          # decreasing radii
        (r, 0, 12, 0.0, 0.0, 4),                # no cells
        (r, 4, 12, 0.9, 0.0, 4),                # buffer >= pi/4
        (r, 4, 12, 0.0, -0.1, 4),               # negative buffer
        (r, 4, 12, 0.0, 0.0, 81),               # l_max above 80
        (np.array([-1.0, 0.5, 1.0]), 4, 12, 0.0, 0.0, 2),   # negative radius
    ]
    for args in bad:
        st, h = yy.yy_grid_create(*args)
        assert st == yy.YY_ERR_INVALID_ARG and not h, args
    for args in [(r[::-1], 4, 12, 4), (r, 4, 0, 4), (r, 4, 12, 81), (np.array([-1.0, 0.5, 1.0]), 4, 12, 2)]:
        st, h = yy.yy_polar_grid_create(*args)
        assert st == yy.YY_ERR_INVALID_ARG and not h, args
    assert yy.yy_potential(None, 16, 16, 16, 16) == yy.YY_ERR_INVALID_ARG
    assert yy.yy_grid_prepare(None, yy.YY_FP64) == yy.YY_ERR_INVALID_ARG
    assert yy.yy_grid_prepare(None, yy.YY_FP64_OZAKI) == yy.YY_ERR_INVALID_ARG
    assert yy.yy_grid_set_analysis(None, yy.YY_ANALYSIS_DENSE) == yy.YY_ERR_INVALID_ARG
    assert yy.yy_last_device_status(None) == yy.YY_ERR_INVALID_ARG
    yy.yy_destroy(None)


def test_binding_constants_match_header():
    """Every enumerator of include/yy.h that the Python binding names has the
    header's value (precisions, statuses, tables, evaluations)."""
    from paper_1806_04593_gb300 import yy
    text = open(os.path.join(ROOT, "include", "yy.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    values = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(YY_[A-Z0-9_]+)\s*=\s*(\d+)", text)}
    assert values["YY_FP64_OZAKI"] == 5
    shared = [n for n in values if hasattr(yy, n)]
    assert len(shared) >= 15
    for name in shared:
        assert getattr(yy, name) == values[name], name
    assert yy.PRECISIONS["fp64_ozaki"] == values["YY_FP64_OZAKI"]
