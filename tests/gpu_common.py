"""Helpers of the GPU tests: build/load the library, run solves through the
C ABI, and compare with the oracle."""

from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


_BUILT = False


def lib():
    global _BUILT
    from paper_1806_04593_gb300 import build, yy
    if not _BUILT:
        build.build()
        _BUILT = True
    yy.load()
    return yy


_FORM = {"prec": None}


def gpu_solve(grid, rho_yin, rho_yang, gradient=False, prec="fp64", stream=None):
    _FORM["prec"] = prec
    dev = torch.device("cuda", 0)
    ry = torch.as_tensor(np.ascontiguousarray(rho_yin), dtype=torch.float64, device=dev)
    rg = torch.as_tensor(np.ascontiguousarray(rho_yang), dtype=torch.float64, device=dev)
    out = grid.solve(ry, rg, gradient=gradient, prec=prec, stream=stream)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def rel_max(a, ref):
    """Normwise max error: max |a - ref| / max |ref|."""
    return float(np.abs(a - ref).max() / np.abs(ref).max())


def rel_l2(a, ref):
    return float(np.linalg.norm((a - ref).ravel()) / np.linalg.norm(ref.ravel()))


def rel_pointwise(a, ref):
    """Pointwise max error: max over cells of |a - ref| / |ref|.  The norm for
    Phi, which is negative at every cell of a positive density; on a steep
    profile |Phi| spans orders of magnitude over r, and a normwise figure
    would hide the error at the outer shells."""
    ref = np.asarray(ref)
    assert np.all(ref != 0.0), "pointwise error needs a reference without zeros"
    return float((np.abs(np.asarray(a) - ref) / np.abs(ref)).max())


def _record(kind, value, l2):
    """Appends a measured error to the file named by YY_ERRLOG (one JSON line
    per check, with the current test id), so that the tolerances below can be
    compared with what a run measured."""
    path = os.environ.get("YY_ERRLOG")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps({"test": os.environ.get("PYTEST_CURRENT_TEST", "?"), "kind": kind,
                                 "value": value, "l2": l2, "prec": _FORM["prec"]}) + "\n")


def phi_err(a, ref):
    """Error of Phi: the pointwise max relative error (also checks that the
    relative L2 error is no larger, which holds for any field)."""
    v = rel_pointwise(a, ref)
    l2 = rel_l2(np.asarray(a), np.asarray(ref))
    _record("phi_pointwise", v, l2)
    assert l2 <= v * (1.0 + 1e-12) + 1e-300
    return v


def grad_err(a, ref):
    """Error of -grad Phi: normwise, max |a - ref| / max |ref| (the field
    vanishes at the centre, so a pointwise ratio is undefined there)."""
    v = rel_max(np.asarray(a), np.asarray(ref))
    _record("grad_normwise", v, rel_l2(np.asarray(a), np.asarray(ref)))
    return v


def field_err(key, a, ref):
    """phi_err for a Phi array ("phi..." keys), grad_err for a gradient."""
    return phi_err(a, ref) if key.startswith("phi") else grad_err(a, ref)


def K_lm(N):
    """K_lm from the oracle's N^(lm): 4 pi / (2l+1) K^2 = N."""
    L = N.shape[0] - 1
    l = np.arange(L + 1)[:, None]
    return np.sqrt((2 * l + 1) / (4 * math.pi) * N)


def mode_index(lmax):
    """List of (l, m, kind) in the library's mode order (kind 'c' or 's')."""
    out = []
    for l in range(lmax + 1):
        out.append((l, 0, "c"))
        for m in range(1, l + 1):
            out.append((l, m, "c"))
            out.append((l, m, "s"))
    return out
