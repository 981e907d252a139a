"""Homogeneous-ellipsoid validation of §5 as a sweep (run by hand on a GPU).

The ellipsoid has semi-axes a = 0.5, b = 1.5 a, c = 2 a and unit density; its
frame is the global one turned by pi/8 about z.  Grids as in §5: equidistant
radial zones on [0, c], "LR" with 400 zones and 2-degree cells, "HR" with
800 zones and 1-degree cells, each as a Yin-Yang grid and as a full
spherical polar grid.  For every l_max the float64 solve (and, at chosen
l_max, the FP16X2 form and the float64 results by the Ozaki scheme) is
compared with the semi-analytic potential at the
solver's output points (r_n^+, cell centres); reported are the maximum and
the L2 relative error over all cells of all patches.

    python -m tests.ellipsoid_sweep --res LR,HR --lmax 0,5,10,20,40,60,80 --out ellipsoid.json
"""

from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

AXES = (0.5, 0.75, 1.0)
DPHI = math.pi / 8
RES = {"LR": (400, 2.0), "HR": (800, 1.0)}


def grid_specs(res):
    from paper_1806_04593_gb300 import inputs
    n_r, deg = RES[res]
    r = np.linspace(0.0, AXES[2], n_r + 1)
    n_t, n_p = int(round(90 / deg)), int(round(270 / deg))
    yy_spec = inputs.GridSpec(f"ellipsoid_{res}_yy", r, n_t, n_p, 0.0, 0.0, 0)
    polar_spec = inputs.polar_grid(r, int(round(180 / deg)), int(round(360 / deg)), 0, f"ellipsoid_{res}_polar")
    return {"yinyang": yy_spec, "polar": polar_spec}


def reference(spec):
    """Cell-averaged densities and the semi-analytic Phi at the output points."""
    from oracle import ellipsoid as el
    from paper_1806_04593_gb300 import inputs
    rho = inputs.ellipsoid_density(spec, AXES, 1.0, DPHI)
    _, units = inputs.cell_centres(spec)
    phi = {p: el.ellipsoid_potential_on_grid(spec.r_edges[1:], units[p], AXES, DPHI) for p in units}
    return rho, phi


def errors(got, ref):
    num = max(float(np.abs(got[p] / ref[p] - 1).max()) for p in ref)
    l2 = math.sqrt(sum(float(((got[p] - ref[p]) ** 2).sum()) for p in ref)
                   / sum(float((ref[p] ** 2).sum()) for p in ref))
    return num, l2


def solve(spec, lmax, rho, prec):
    import dataclasses

    import torch

    from paper_1806_04593_gb300 import yy
    dev = torch.device("cuda", 0)
    g = yy.Grid.from_spec(dataclasses.replace(spec, lmax=lmax))
    try:
        if prec != "fp64":
            g.prepare(prec)
        ry = torch.as_tensor(rho[0], device=dev)
        if spec.polar:
            out = {"yin": g.solve(ry, prec=prec)["phi"]}
        else:
            res = g.solve(ry, torch.as_tensor(rho[1], device=dev), prec=prec)
            out = {"yin": res["phi_yin"], "yang": res["phi_yang"]}
        torch.cuda.synchronize()
        return {p: v.cpu().numpy() for p, v in out.items()}
    finally:
        g.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--res", default="LR,HR")
    ap.add_argument("--lmax", default="0,5,10,20,40,60,80")
    ap.add_argument("--fp16x2-at", default="20,40")
    ap.add_argument("--ozaki-at", default="20")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    from paper_1806_04593_gb300 import build
    build.build()
    lmaxes = [int(v) for v in args.lmax.split(",")]
    half = {int(v) for v in args.fp16x2_at.split(",") if v}
    oz = {int(v) for v in args.ozaki_at.split(",") if v}
    rows = []
    for res in args.res.split(","):
        for kind, spec in grid_specs(res).items():
            t0 = time.time()
            rho, ref = reference(spec)
            t_ref = time.time() - t0
            for L in lmaxes:
                for prec in ["fp64"] + (["fp16x2"] if L in half else []) + (["fp64_ozaki"] if L in oz else []):
                    t1 = time.time()
                    got = solve(spec, L, rho, prec)
                    e_max, e_l2 = errors(got, ref)
                    row = {"res": res, "grid": kind, "l_max": L, "prec": prec, "rel_max": e_max,
                           "rel_l2": e_l2, "solve_s": time.time() - t1, "reference_s": t_ref}
                    rows.append(row)
                    print(json.dumps(row), flush=True)
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(rows, fh, indent=1)


if __name__ == "__main__":
    main()
