"""Timing of the CPU float64 oracle on the host cores (run by hand).

For the tiny, mid and production grids and four fields of the batched
workload, one solve with -grad Phi, once with one thread and once with all
cores (the BLAS thread count is fixed per child process through the usual
environment variables).  Grid construction (the paper's constant terms) is
timed separately.  Large grids evaluate a sample of the target cells and
scale that part of the time; the sample is stated per row.

    python -m tests.oracle_timing --out oracle_timing.json
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [("tiny", 1), ("mid", 1), ("production", 16)] + [(f"batched{f}", 8) for f in range(4)]


def child(case, div):
    sys.path.insert(0, ROOT)
    import numpy as np

    from oracle import OracleGrid
    from paper_1806_04593_gb300 import inputs
    if case.startswith("batched"):
        spec, seed, eps = inputs.batched_specs()[int(case[len("batched"):])]
        ry, rg = inputs.pns_density(spec, seed, eps)
    else:
        spec = inputs.GRIDS[case]()
        ry, rg = inputs.density_for(spec)
    t0 = time.perf_counter()
    og = OracleGrid(spec.r_edges, spec.n_theta, spec.n_phi, spec.delta_theta, spec.delta_phi, spec.lmax, spec.G)
    t_create = time.perf_counter() - t0
    cells = np.arange(0, spec.n_ang, div) if div > 1 else None
    # the density-dependent part that does not scale with the cells: analysis and radial sums
    t0 = time.perf_counter()
    og.radial_sums(*og.analysis(ry))
    og.radial_sums(*og.analysis(rg))
    t_fixed = time.perf_counter() - t0
    t0 = time.perf_counter()
    og.solve(ry, rg, gradient=True, cells=cells)
    t_solve = time.perf_counter() - t0
    n_cells = spec.n_ang if cells is None else cells.size
    t_full = t_fixed + (t_solve - t_fixed) * spec.n_ang / n_cells
    print(json.dumps({"case": case, "n_r": spec.n_r, "n_theta": spec.n_theta, "n_phi": spec.n_phi,
                      "l_max": spec.lmax, "create_s": t_create, "solve_s": t_full,
                      "sample": f"1/{div} of the cells" if div > 1 else "all cells"}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--child", nargs=2, default=None)
    args = ap.parse_args()
    if args.child:
        child(args.child[0], int(args.child[1]))
        return
    cores = os.cpu_count()
    rows = []
    for case, div in CASES:
        for threads in (1, cores):
            env = dict(os.environ)
            for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
                env[k] = str(threads)
            res = subprocess.run([sys.executable, "-m", "tests.oracle_timing", "--child", case, str(div)],
                                 cwd=ROOT, env=env, capture_output=True, text=True, check=True)
            row = json.loads(res.stdout.strip().splitlines()[-1])
            row["threads"] = threads
            row["solves_per_s"] = 1.0 / row["solve_s"]
            rows.append(row)
            print(json.dumps(row), flush=True)
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(rows, fh, indent=1)


if __name__ == "__main__":
    main()
