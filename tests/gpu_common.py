"""Helpers of the GPU tests: build/load the library, run solves through the
C ABI, and compare with the oracle."""

from __future__ import annotations

import math

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


def gpu_solve(grid, rho_yin, rho_yang, gradient=False, prec="fp64", stream=None):
    dev = torch.device("cuda", 0)
    ry = torch.as_tensor(np.ascontiguousarray(rho_yin), dtype=torch.float64, device=dev)
    rg = torch.as_tensor(np.ascontiguousarray(rho_yang), dtype=torch.float64, device=dev)
    out = grid.solve(ry, rg, gradient=gradient, prec=prec, stream=stream)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def rel_max(a, ref):
    return float(np.abs(a - ref).max() / np.abs(ref).max())


def rel_l2(a, ref):
    return float(np.linalg.norm((a - ref).ravel()) / np.linalg.norm(ref.ravel()))


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
