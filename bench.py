#!/usr/bin/env python3
"""Benchmark of the Yin-Yang multipole gravity solver on GB300.

Workload: the 1-degree Yin-Yang grid (90 x 270 cells per patch), 550
log-spaced zones in [1e-4, 1], l_max = 25, with the seeded proto-neutron-star
density; tables prebuilt.  One step = one solve of Phi and -grad Phi on both
patches (analysis, radial scans, synthesis).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec P] [--impl ours|reference]

Prints one JSON line (rank 0).  The headline is float64 accuracy:
YY_FP64_OZAKI by default (float64 results, the azimuthal stages as exact
digit products on the tensor cores), within 1e-12 of the float64 oracle.
`value` is solves/s over all ranks from device-side CUDA events, L2 flushed
before every step; `e2e` is the same metric through the host-buffer entry
points (pinned host buffers, host<->device copies inside the timed region).
`forms` times every other arithmetic form (FP16X2, BF16X3, TF32, FP32 and the
plain float64 CUDA-core path) the same way, each with its error against the
float64 oracle over all cells (Phi pointwise, -grad Phi normwise).
`kernels_ms` lists the headline's kernels as timed by the library's CUDA
events on the solve's stream; `roofline` is that of the longest one.  The
`batched` object times the 64-field workload (one CUDA graph per step) in
the mixed-precision form of that workload.  With several GPUs every rank
solves its own field (replicas, weak scaling).  The reference arm times the
CPU float64 oracle, full solves, on the host cores.
"""

from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "YY Poisson solves/s and GEMM TFLOP/s (1° grid, l_max=25) at stated rel. error vs FP64"
UNIT = "solves/s"
L2_BYTES = 126 * 1024 * 1024
# float64 pipe of GB300: 152 SMs x 2 DFMA per clock x 2 flop x 2070 MHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# fp32 pipe: 152 SMs x 128 FFMA per clock x 2 flop x 2070 MHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# fp32 operations of one float-float multiply-add (TwoProduct by FMA with the
# cross terms, TwoSum into the high part, the low parts added)
FF_OPS = 12
FORMS = ("fp64_ozaki", "fp16x2", "bf16x3", "tf32", "fp32", "fp64")
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16x2": "fp16x2 (fp32 accumulate, f64 scans)",
         "bf16x3": "bf16x3 (fp32 accumulate, f64 scans)", "tf32": "tf32 (fp32 accumulate, f64 scans)",
         "fp64_ozaki": "f64"}
PRODUCTS = {"fp16x2": 3, "bf16x3": 6, "tf32": 1}

# DRAM bytes (read + write) per launch of a kernel, from one ncu capture of
# this workload (profiles/), valid only while the kernel sources are the ones
# captured, up to comments and blank lines (digest of
# paper_1806_04593_gb300/csrc with both removed).
_TRAFFIC = {"k_oz_synth": (333.456128 + 807.069952) * 1e6}
_TRAFFIC_SRC = "83b880329c4d8cfc950ee4b606c675270d0796c835530a7ed5adcda23ce878fa"

_COMMENT = re.compile(rb"/\*.*?\*/|//[^\n]*", re.S)


def _code_only(src):
    """C/C++/CUDA source without its comments, trailing blanks and blank lines
    (the sources hold no string literal with // or /* in it)."""
    lines = (ln.rstrip() for ln in _COMMENT.sub(b"", src).split(b"\n"))
    return b"\n".join(ln for ln in lines if ln)


def _csrc_digest():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1806_04593_gb300", "csrc")
    for fn in sorted(os.listdir(d)):
        if fn.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(d, fn), "rb") as fh:
                h.update(fn.encode() + b"\0" + _code_only(fh.read()))
    return h.hexdigest()


def _recorded_traffic(kernel):
    if _TRAFFIC_SRC is None or kernel not in _TRAFFIC:
        return None
    return _TRAFFIC[kernel] if _csrc_digest() == _TRAFFIC_SRC else None


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        p.setdefault("source", "measured (MEASURED_PEAKS.json)")
        return p
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "source": "fallback (no MEASURED_PEAKS.json)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp64_ozaki", choices=FORMS + ("auto",))
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the other arithmetic forms")
    ap.add_argument("--form-steps", type=int, default=20)
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-field batched workload")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--batch-profile", type=int, default=None, metavar="GROUPS",
                    help="after the batch timing, replay its graph once inside cudaProfilerStart/Stop "
                         "(ncu --profile-from-start off) in this form: 0 per-field graph, N >= 1 grouped")
    ap.add_argument("--ref-budget-s", type=float, default=240.0,
                    help="reference arm: full oracle solves per step while (steps + warmup) fit in this time")
    ap.add_argument("--ref-cells-div", type=int, default=0,
                    help="reference arm: evaluate 1/D of the cells per step (D > 1; 0 = decide by the budget)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only: a barrier and a max over ranks)
# ---------------------------------------------------------------------------

class Dist:
    def __init__(self, init=True):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1 and init:
            import torch.distributed as dist
            backend = "nccl" if self._cuda() else "gloo"
            dist.init_process_group(backend)
            self.pg = dist

    @staticmethod
    def _cuda():
        import torch
        return torch.cuda.is_available()

    def barrier(self):
        if self.pg:
            import torch
            if self._cuda():
                self.pg.barrier(device_ids=[self.local])
            else:
                self.pg.barrier()

    def max(self, x):
        if not self.pg:
            return x
        import torch
        t = torch.tensor([float(x)], device="cuda" if self._cuda() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "20"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # wait (at most 5 s) for the first sample, so that sampling covers the timed region
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None:
            self.fh.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


# ---------------------------------------------------------------------------
# errors against the float64 oracle
# ---------------------------------------------------------------------------

def field_errors(got, ref, gradient):
    """Phi: pointwise max |dPhi|/|Phi| (Phi < 0 at every cell) and relative L2;
    -grad Phi: normwise max |dg|/max|g| and relative L2 (g vanishes at the centre)."""
    import numpy as np
    out = {}
    for key in ("phi_yin", "phi_yang") + (("grad_yin", "grad_yang") if gradient else ()):
        a, r = np.asarray(got[key]), np.asarray(ref[key])
        d = np.abs(a - r)
        e = {"rel_l2": float(np.linalg.norm(d) / np.linalg.norm(r)),
             "rel_max_normwise": float(d.max() / np.abs(r).max())}
        if key.startswith("phi"):
            e["rel_max_pointwise"] = float((d / np.abs(r)).max())
        out[key] = e
    phi = max(out[k]["rel_max_pointwise"] for k in ("phi_yin", "phi_yang"))
    summary = {"phi_rel_max_pointwise": phi,
               "phi_rel_l2": max(out[k]["rel_l2"] for k in ("phi_yin", "phi_yang"))}
    if gradient:
        summary["grad_rel_max_normwise"] = max(out[k]["rel_max_normwise"] for k in ("grad_yin", "grad_yang"))
        summary["grad_rel_l2"] = max(out[k]["rel_l2"] for k in ("grad_yin", "grad_yang"))
    summary["fields"] = out
    return summary


# ---------------------------------------------------------------------------
# the oracle (cpu_baseline and the reference arm): full solves, measured
# ---------------------------------------------------------------------------

def oracle_grid(spec):
    from oracle import OracleGrid
    return OracleGrid(spec.r_edges, spec.n_theta, spec.n_phi, spec.delta_theta, spec.delta_phi, spec.lmax, spec.G)


def _single_thread_oracle(gradient, sample_div):
    """The oracle with one BLAS / OpenMP thread, in a child process (the
    thread count of numpy's BLAS is fixed when it loads): analysis and radial
    sums of both patches in full, the evaluation at 1/sample_div of the cells,
    that part scaled to all cells."""
    code = (
        "import json, sys, time\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import numpy as np\n"
        "from paper_1806_04593_gb300 import inputs\n"
        "from oracle import OracleGrid\n"
        "spec = inputs.production_grid()\n"
        "ry, rg = inputs.density_for(spec)\n"
        "og = OracleGrid(spec.r_edges, spec.n_theta, spec.n_phi, spec.delta_theta, spec.delta_phi, spec.lmax, spec.G)\n"
        "t0 = time.perf_counter()\n"
        "for rho in (ry, rg): og.radial_sums(*og.analysis(rho))\n"
        "fixed = time.perf_counter() - t0\n"
        f"cells = np.arange(0, spec.n_ang, {sample_div})\n"
        "t0 = time.perf_counter()\n"
        f"og.solve(ry, rg, gradient={bool(gradient)}, cells=cells)\n"
        "t = time.perf_counter() - t0\n"
        "print(json.dumps({'fixed': fixed, 'sample': t, 'cells': int(cells.size), 'n_ang': spec.n_ang}))\n")
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    try:
        res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        rec = json.loads(res.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError) as exc:
        return {"unavailable": f"single-thread oracle run failed: {exc}"}
    # the sample solve repeats the full analysis and radial sums once
    eval_s = max(rec["sample"] - rec["fixed"], 0.0) * rec["n_ang"] / rec["cells"]
    t = rec["fixed"] + eval_s
    return {"value": 1.0 / t, "unit": UNIT, "cores": 1, "extrapolated": True,
            "sample": (f"one BLAS thread: analysis + radial sums of both patches in full ({rec['fixed']:.2f} s), "
                       f"the evaluation at 1/{sample_div} of the cells ({rec['cells']} cells x all radii), "
                       f"that part scaled x{rec['n_ang'] / rec['cells']:.0f}")}


def cpu_baseline(spec, ry, rg, gradient):
    """One full oracle solve on every host core (measured), and the
    single-thread rate beside it.  Returns (info, full-field result)."""
    og = oracle_grid(spec)
    t0 = time.perf_counter()
    ref = og.solve(ry, rg, gradient=gradient)
    t = time.perf_counter() - t0
    info = {"value": 1.0 / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"one full solve of the workload (all {spec.n_ang} cells x {spec.n_r} radii per patch, "
                       f"Phi{' and -grad Phi' if gradient else ''}), numpy float64 oracle, BLAS on all "
                       f"{os.cpu_count()} host cores, tables prebuilt: {t:.2f} s measured"),
            "single_thread": _single_thread_oracle(gradient, 16)}
    return info, ref


# ---------------------------------------------------------------------------
# algorithmic work per kernel (roofline)
# ---------------------------------------------------------------------------

def kernel_work(name, spec, n_lm, gradient, prec):
    """Algorithmic work of one launch of a named kernel of the solve:
    {"flop": ..., "flop_kind": "tensor"|"fp64"|"fp32", "bytes": ...} (the
    entries that apply), each counted from the sizes of the workload."""
    L = spec.lmax
    n_r2 = 2 * spec.n_r                       # rows of both patches
    J = 4 if gradient else 1                  # Phi and the three gradient components
    nt = 2 * L + 1
    half = (spec.n_theta + 1) // 2
    rows = n_r2 * spec.n_theta                # (shell, theta row) rows of the separable stages
    f64 = 8
    out_bytes = J * n_r2 * spec.n_ang * f64
    w = {}
    if name.startswith("k_tc_pair<FormOzaki,3>/synthesis") or name == "k_oz_synth":
        k_pad = -(-nt // 32) * 32
        w = {"flop": 2.0 * rows * spec.n_phi * nt * J, "flop_kind": "tensor", "products": "ozaki",
             "bytes": out_bytes + J * rows * k_pad * 6 * 2}
    elif name.startswith("k_tc_pair<FormOzaki,3>/analysis") or name == "k_oz_analysis":
        k_pad = -(-spec.n_phi // 64) * 64
        w = {"flop": 2.0 * rows * spec.n_phi * nt, "flop_kind": "tensor", "products": "ozaki",
             "bytes": rows * k_pad * 6 * 2}
    elif name == "k_theta_ff":
        # float-float multiply-adds of Phi, g_r and g_theta (g_phi is formed
        # from Phi's sums), one per term and mirrored row pair
        ffma = sum(L + 1 - (t + 1) // 2 for t in range(nt)) * min(J, 3)
        gk = 64 if nt <= 64 else 128
        w = {"flop": 2.0 * n_r2 * half * ffma, "flop_kind": "ff",
             "bytes": J * rows * gk * 6 * 2 + min(J, 3) * n_r2 * n_lm * f64}
    elif name == "k_q_ff":
        w = {"bytes": 2 * min(J, 3) * n_r2 * n_lm * f64}
    elif name == "k_rhow_ozaki":
        k_pad = -(-spec.n_phi // 64) * 64
        w = {"bytes": n_r2 * spec.n_ang * f64 + rows * k_pad * 6 * 2}
    elif name == "k_sep_theta_ff":
        nt_pad = -(-nt // 4) * 4
        w = {"flop": 2.0 * n_r2 * n_lm * half, "flop_kind": "ff",
             "bytes": rows * nt_pad * f64 + n_r2 * n_lm * f64}
    elif name.startswith("k_sep_theta"):
        w = {"flop": 2.0 * n_r2 * n_lm * half, "flop_kind": "fp64" if "double" in name or prec == "fp64" else "fp32",
             "bytes": rows * (-(-nt // 4) * 4) * f64 + n_r2 * n_lm * f64}
    elif name == "k_scan_warp":
        w = {"bytes": n_r2 * n_lm * f64 * 4}
    elif name == "k_rotate_moments":
        s = sum((2 * l + 1) ** 2 for l in range(L + 1))
        w = {"flop": 2.0 * n_r2 * s, "flop_kind": "fp64", "bytes": 3 * n_r2 * n_lm * f64}
    elif name == "k_tc_pair/synthesis":
        w = {"flop": 2.0 * n_r2 * n_lm * spec.n_ang * J, "flop_kind": "tensor", "products": prec,
             "bytes": out_bytes}
    elif name == "k_tc_pair/split-K":
        w = {"flop": 2.0 * n_r2 * n_lm * spec.n_ang, "flop_kind": "tensor", "products": prec}
    elif name == "k_pack_stream":
        w = {"bytes": n_r2 * spec.n_ang * f64 + n_r2 * spec.n_ang * {"fp16x2": 4, "bf16x3": 6, "tf32": 4}.get(prec, 4)}
    elif name == "k_sep_synth":
        w = {"flop": J * (2.0 * rows * n_lm + 2.0 * rows * spec.n_phi * nt),
             "flop_kind": "fp64" if prec == "fp64" else "fp32", "bytes": out_bytes}
    elif name == "k_sep_phi":
        w = {"flop": 2.0 * rows * spec.n_phi * nt, "flop_kind": "fp64" if prec == "fp64" else "fp32",
             "bytes": n_r2 * spec.n_ang * f64}
    return w


def roofline_of(name, ms, spec, n_lm, gradient, prec, peaks, ozaki_products):
    """Roofline object of one kernel from its event-timed duration: the
    binding resource (the larger fraction of peak) with the other beside it."""
    w = kernel_work(name, spec, n_lm, gradient, prec)
    s = ms / 1e3
    cands = []
    if "flop" in w:
        kind = w["flop_kind"]
        if kind == "tensor":
            prods = ozaki_products if w.get("products") == "ozaki" else PRODUCTS.get(w.get("products"), 1)
            ratio = 0.5 if prec == "tf32" and w.get("products") != "ozaki" else 1.0
            hw = w["flop"] * prods
            cands.append({"bound": "tensor", "achieved": hw / s / 1e12, "peak": peaks["bf16_tflops"] * ratio,
                          "unit": "TFLOP/s",
                          "work": (f"hardware products: {prods} x 2MNK = {hw / 1e9:.1f} GFLOP per launch "
                                   f"(algorithmic float64 work {w['flop'] / 1e9:.2f} GFLOP)"),
                          "peak_source": ("measured bf16 burst" + (" x 0.5 (tf32 nominal ratio)" if ratio < 1 else "")
                                          + f", {peaks['source']}")})
        elif kind == "ff":
            cands.append({"bound": "alu", "achieved": w["flop"] / s / 1e12, "peak": FP32_PEAK_TFLOPS / FF_OPS,
                          "unit": "TFLOP/s",
                          "work": f"float-float multiply-adds x 2 = {w['flop'] / 1e9:.2f} GFLOP per launch",
                          "peak_source": (f"derived: 152 SMs x 128 FFMA per clock x 2 flop x 2070 MHz, divided by "
                                          f"the {FF_OPS} fp32 operations of one float-float multiply-add")})
        else:
            peak = FP64_PEAK_TFLOPS if kind == "fp64" else FP32_PEAK_TFLOPS
            cands.append({"bound": "alu", "achieved": w["flop"] / s / 1e12, "peak": peak, "unit": "TFLOP/s",
                          "work": f"{kind} multiply-adds x 2 = {w['flop'] / 1e9:.2f} GFLOP per launch",
                          "peak_source": (f"derived: 152 SMs x {'2 DFMA' if kind == 'fp64' else '128 FFMA'} "
                                          "per clock x 2 flop x 2070 MHz")})
    if "bytes" in w:
        cands.append({"bound": "hbm", "achieved": w["bytes"] / s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                      "work": f"algorithmic bytes {w['bytes'] / 1e6:.1f} MB per launch",
                      "peak_source": f"measured copy bandwidth, {peaks['source']}"})
    if not cands:
        return {"kernel": name, "bound": None, "ms": ms}
    for c in cands:
        c["frac"] = c["achieved"] / c["peak"]
    cands.sort(key=lambda c: -c["frac"])
    best = dict(cands[0])
    best.update(kernel=name, ms=ms, traffic=_recorded_traffic(name))
    if len(cands) > 1:
        best["other"] = cands[1]
    return best


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def timed_steps(step, steps, warmup, stream, flush):
    """W untimed steps, then K steps each bracketed by CUDA events on the
    solve's stream, L2 flushed (a 252 MB write) before each.  The host
    enqueues every step without waiting, as a caller's loop would."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)]


def profile_kernels(yy, grid, step, steps, flush):
    """Per-stage and per-kernel times (the library's CUDA events on the
    solve's stream), averaged over `steps` solves; reading them synchronises
    after each solve, so this pass is kept apart from the timed loop."""
    stage_tot = {k: 0.0 for k in yy.STAGES}
    kern = {}
    yy.yy_grid_set_profiling(grid.handle, 1)
    for _ in range(steps):
        flush.zero_()
        step()
        st, stages = yy.yy_grid_stage_ms(grid.handle)
        for k in stage_tot:
            stage_tot[k] += stages[k]
        seen = {}
        for name, ms in yy.yy_grid_kernels_ms(grid.handle):
            n = seen.get(name, 0)
            seen[name] = n + 1
            key = name if n == 0 else f"{name}#{n + 1}"
            kern[key] = kern.get(key, 0.0) + ms
    yy.yy_grid_set_profiling(grid.handle, 0)
    return ({k: v / steps for k, v in stage_tot.items()}, {k: v / steps for k, v in kern.items()})


def run_ours(args, dist):
    import numpy as np
    import torch

    from paper_1806_04593_gb300 import build as yybuild
    from paper_1806_04593_gb300 import inputs, yy

    if dist.rank == 0:
        yybuild.build()
    dist.barrier()
    yy.load()
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    stream = torch.cuda.current_stream(dev)
    gradient = not args.no_grad
    peaks = _measured_peaks()

    spec = inputs.production_grid()
    grid = yy.Grid.from_spec(spec)
    prec = "fp64_ozaki" if args.prec == "auto" else args.prec
    grid.prepare(prec)
    ry_np, rg_np = inputs.density_for(spec)
    ry = torch.from_numpy(ry_np).to(dev)
    rg = torch.from_numpy(rg_np).to(dev)
    shape = grid.field_shape
    phi_y = torch.empty(shape, dtype=torch.float64, device=dev)
    phi_g = torch.empty_like(phi_y)
    g_y = torch.empty((3,) + shape, dtype=torch.float64, device=dev) if gradient else None
    g_g = torch.empty_like(g_y) if gradient else None
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def solver(form):
        def step():
            grid.potential(ry, rg, phi_y, phi_g, g_y, g_g, prec=form, stream=stream)
        return step

    def outputs():
        o = {"phi_yin": phi_y.cpu().numpy(), "phi_yang": phi_g.cpu().numpy()}
        if gradient:
            o["grad_yin"], o["grad_yang"] = g_y.cpu().numpy(), g_g.cpu().numpy()
        return o

    solve = solver(prec)
    solve()
    torch.cuda.synchronize()
    launches = yy.yy_last_launch_count(grid.handle)

    # ---- headline: device-timed region with clocks sampled
    clocks = ClockSampler(dist.local)
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    w0 = time.perf_counter()
    step_ms = timed_steps(solve, args.steps, args.warmup, stream, flush)
    wall = time.perf_counter() - w0
    dist.barrier()
    clk = clocks.stop()
    dev_s_max = dist.max(sum(step_ms) / 1e3)
    value = dist.world * args.steps / dev_s_max
    stage_ms, kernels_ms = profile_kernels(yy, grid, solve, min(args.steps, 20), flush)
    solve()
    torch.cuda.synchronize()
    assert yy.yy_last_device_status(grid.handle) == yy.YY_OK
    headline_out = outputs()

    # ---- end to end through the host-buffer entry points
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_ry, h_rg = pin(ry_np), pin(rg_np)
    mk = lambda shp: torch.empty(shp, dtype=torch.float64).pin_memory()
    h_out = [tuple([mk(shape), mk(shape)] + ([mk((3,) + shape), mk((3,) + shape)] if gradient else [None, None]))
             for _ in range(2)]
    pcode = yy.PRECISIONS[prec]
    e2e_steps = min(args.steps, 50)
    for _ in range(max(1, args.warmup // 2)):
        yy.yy_potential_host(grid.handle, h_ry, h_rg, *h_out[0], pcode, stream)
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        st = yy.yy_potential_host(grid.handle, h_ry, h_rg, *h_out[0], pcode, stream)
        assert st == yy.YY_OK, yy.yy_status_string(st)
    e2e_sync_s = dist.max(time.perf_counter() - t0) / e2e_steps
    for i in range(2):
        yy.yy_potential_host_async(grid.handle, h_ry, h_rg, *h_out[i % 2], pcode, stream)
    yy.yy_potential_host_wait(grid.handle)
    dist.barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        st = yy.yy_potential_host_async(grid.handle, h_ry, h_rg, *h_out[i % 2], pcode, stream)
        assert st == yy.YY_OK, yy.yy_status_string(st)
    st = yy.yy_potential_host_wait(grid.handle)
    assert st == yy.YY_OK, yy.yy_status_string(st)
    e2e_s = dist.max(time.perf_counter() - t0) / e2e_steps
    field_bytes = ry_np.nbytes
    h2d = 2 * field_bytes
    d2h = 2 * field_bytes + (6 * field_bytes if gradient else 0)

    # ---- roofline of the headline's longest kernel (library events on the stream)
    oz_products = 26
    top = max(kernels_ms, key=kernels_ms.get)
    roof = roofline_of(top.split("#")[0], kernels_ms[top], spec, grid.n_lm, gradient, prec, peaks, oz_products)
    kernel_roofs = {k: roofline_of(k.split("#")[0], v, spec, grid.n_lm, gradient, prec, peaks, oz_products)
                    for k, v in kernels_ms.items()}

    # ---- the float64 oracle: one full solve on the host cores (rank 0, N = 1)
    ref = None
    cpu = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        cpu, ref = cpu_baseline(spec, ry_np, rg_np, gradient)

    # ---- every other arithmetic form, timed the same way
    forms = {}
    if not args.no_forms:
        for form in FORMS:
            if form == prec:
                continue
            try:
                grid.prepare(form)
            except yy.YYError as exc:
                forms[form] = {"unavailable": str(exc)}
                continue
            step = solver(form)
            step()
            torch.cuda.synchronize()
            ms = timed_steps(step, args.form_steps, 3, stream, flush)
            f_stage, f_kern = profile_kernels(yy, grid, step, 5, flush)
            step()
            torch.cuda.synchronize()
            assert yy.yy_last_device_status(grid.handle) == yy.YY_OK
            got = outputs()
            ms_mean = sum(ms) / len(ms)
            rec = {"value": 1e3 / ms_mean, "unit": UNIT, "ms_per_step": ms_mean, "steps": args.form_steps,
                   "dtype": DTYPE[form], "stage_ms": f_stage, "kernels_ms": f_kern,
                   "speedup_of_headline": ms_mean / (sum(step_ms) / len(step_ms))}
            ftop = max(f_kern, key=f_kern.get)
            rec["roofline"] = roofline_of(ftop.split("#")[0], f_kern[ftop], spec, grid.n_lm, gradient, form, peaks,
                                          oz_products)
            if ref is not None:
                rec["error_vs_fp64_oracle"] = field_errors(got, ref, gradient)
            else:
                rec["error_vs_headline"] = field_errors(got, headline_out, gradient)
            forms[form] = rec

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dev_s_max * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[prec],
        "data": "synthetic (seeded proto-neutron-star density, l<=4 angular perturbation)",
        "config": {"workload": ("1-degree Yin-Yang grid, 2 x 90 x 270 cells, n_r=550 log r in [1e-4,1], "
                                "l_max=25, " + ("Phi and -grad Phi per solve" if gradient else "Phi only")),
                   "n_r": spec.n_r, "n_theta": spec.n_theta, "n_phi": spec.n_phi, "l_max": spec.lmax,
                   "gradient": gradient, "precision": prec, "parallelism": f"replicas x{dist.world}",
                   "l2": "L2 flushed (252 MB write) before every timed step"},
        "precision_note": ("float64 results: the azimuthal stages of analysis and synthesis as bf16 digit "
                           "products on tcgen05 (48-bit operands, exact per level, rounded once to float64), "
                           "the polar stages in float-float arithmetic on the fp32 pipe (about 48 bits), "
                           "combination and radial scans in float64") if prec == "fp64_ozaki" else None,
        "gemm_tflops": grid.flops(gradient) / (dev_s_max / args.steps) / 1e12,
        "stage_ms": stage_ms,
        "kernels_ms": kernels_ms,
        "kernel_rooflines": kernel_roofs,
        "wall_s": wall,
        "roofline": roof,
        "e2e": {"value": dist.world / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "api": ("yy_potential_host_async (pinned host buffers, copies overlapped across calls), "
                        f"{e2e_steps} calls then yy_potential_host_wait"),
                "synchronous_call": {"value": dist.world / e2e_sync_s, "unit": UNIT,
                                     "api": "yy_potential_host (copy in, solve, copy out, sync per call)"}},
        "gpu_launches": launches * args.steps,
        "clocks": clk,
        "forms": forms,
    }
    if ref is not None:
        out["error_vs_fp64_oracle"] = field_errors(headline_out, ref, gradient)
        out["cpu_baseline"] = cpu
    out["radial_scan_static_us"] = time_static_scan(yy, grid, spec, stream, flush)

    # ---- the batched workload (uneven fields in one graph), rank-local
    if not args.no_batch:
        out["batched"] = run_batched(args, gradient, dev, stream, flush)
    grid.close()
    return out


def time_static_scan(yy, grid, spec, stream, flush):
    """yy_radial_scan_static on the workload's own combined moments (CUDA
    events, L2 flushed before each call), beside the solve's scan kernel."""
    import torch
    dev = flush.device
    moments = torch.from_numpy(grid.table(yy.YY_TABLE_MOMENTS_TOTAL)).to(dev)
    r = torch.from_numpy(spec.r_edges.copy()).to(dev)
    coeff = torch.empty((3, 2 * spec.n_r, grid.n_lm), dtype=torch.float64, device=dev)
    step = lambda: yy.yy_radial_scan_static(r, spec.n_r, spec.lmax, spec.G, moments, coeff, stream)
    if step() != yy.YY_OK:
        return None
    ms = timed_steps(step, 10, 2, stream, flush)
    return 1e3 * sum(ms) / len(ms)


def run_batched(args, gradient, dev, stream, flush):
    """The batched workload: 64 fields of uneven size (n_r ~ U{100..600}, 2 /
    1.5 / 1 degree cells, l_max ~ U{10..40}), in the mixed-precision form
    (FP16X2) with the evaluation of each field picked by yy_batch_tune, all
    solves replayed as one CUDA graph per step; beside it the same batch in
    float64 (CUDA cores) and the error of Phi against that, field by field."""
    import torch

    from paper_1806_04593_gb300 import inputs, yy

    prec = "fp16x2"
    items = inputs.batched_specs()
    specs = [sp for sp, _, _ in items]
    b = yy.Batch(specs)
    t0 = time.perf_counter()
    chosen = b.tune(prec, gradient=gradient, reps=1)
    tune_s = time.perf_counter() - t0
    rho, outs = [], []
    for sp, seed, eps in items:
        ry, rg = inputs.pns_density(sp, seed, eps)
        rho.append((torch.from_numpy(ry).to(dev), torch.from_numpy(rg).to(dev)))
        shape = (sp.n_r, sp.n_theta, sp.n_phi)
        o = [torch.empty(shape, dtype=torch.float64, device=dev) for _ in range(2)]
        if gradient:
            o += [torch.empty((3,) + shape, dtype=torch.float64, device=dev) for _ in range(2)]
        outs.append(o)

    def step(form):
        b.potential([r[0] for r in rho], [r[1] for r in rho], [o[0] for o in outs], [o[1] for o in outs],
                    [o[2] for o in outs] if gradient else None, [o[3] for o in outs] if gradient else None,
                    prec=form, stream=stream)

    def timed(form, steps, warmup):
        ms = timed_steps(lambda: step(form), steps, warmup, stream, flush)
        st = b.device_status()
        assert st == yy.YY_OK, yy.yy_status_string(st)
        return sum(ms) / len(ms)

    ms = timed(prec, args.batch_steps, max(3, args.warmup))
    launches = b.launch_count()
    groups = b.groups()
    # the graph forms the first capture chose between, each timed the same way
    modes = {}
    for ng in (0, 1, 2, 4):
        b.set_grouping(ng)
        m = timed(prec, args.batch_steps, max(3, args.warmup))
        modes["per_field_graph" if ng == 0 else f"grouped_{ng}"] = {
            "ms_per_step": m, "kernels_per_step": b.launch_count(), "value": len(specs) * 1e3 / m}
    b.set_grouping(groups)
    if args.batch_profile is not None:
        # one replay in the given graph form inside the profiler range
        b.set_grouping(args.batch_profile)
        step(prec)
        step(prec)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        step(prec)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        b.set_grouping(groups)
    splits = [b.analysis_splits(i, prec) for i in range(len(specs))]
    # each field solved alone on its own grid (tuned settings), back to back
    solo_ms = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i, (sp, (ry, rg), o) in enumerate(zip(specs, rho, outs)):
        h = b.grid_handle(i)
        args_i = (h, ry, rg, o[0], o[1], o[2] if gradient else None, o[3] if gradient else None,
                  yy.PRECISIONS[prec], stream)
        yy.yy_potential(*args_i)
        e0.record(stream)
        yy.yy_potential(*args_i)
        e1.record(stream)
        torch.cuda.synchronize()
        solo_ms += e0.elapsed_time(e1)
    phi = [(o[0].clone(), o[1].clone()) for o in outs]
    b.prepare("fp64")
    ms64 = timed("fp64", 3, 1)
    err = 0.0
    for (py, pg), o in zip(phi, outs):
        for got, ref in ((py, o[0]), (pg, o[1])):
            err = max(err, float(((got - ref).abs() / ref.abs()).max()))
    ref64 = [[t.clone() for t in o] for o in outs]
    # the same batch at float64 accuracy on the tensor cores (Ozaki digits)
    b.prepare("fp64_ozaki")
    b.tune("fp64_ozaki", gradient=gradient, reps=1)
    ms_oz = timed("fp64_ozaki", args.batch_steps, max(3, args.warmup))
    err_oz = 0.0
    for r, o in zip(ref64, outs):
        for got, ref in ((o[0], r[0]), (o[1], r[1])):
            err_oz = max(err_oz, float(((got - ref).abs() / ref.abs()).max()))
    cells = sum(2 * sp.n_r * sp.n_ang for sp in specs)   # both patches
    res = {
        "workload": "64 fields, n_r ~ U{100..600}, 2 / 1.5 / 1 degree cells, l_max ~ U{10..40}, "
                    "seeded proto-neutron-star densities with eps scale ~ U(0.01, 0.1)",
        "value": len(specs) * 1e3 / ms, "unit": "field solves/s", "ms_per_step": ms,
        "zone_cells_per_s": cells * 1e3 / ms,
        "precision": prec, "gradient": gradient,
        "analysis_chosen": {"dense": chosen.count(yy.YY_ANALYSIS_DENSE),
                            "separable": chosen.count(yy.YY_ANALYSIS_SEPARABLE)},
        "tune_s": tune_s, "graph_launches_per_step": 1, "kernels_per_step": launches,
        "graph_form": (f"{groups} concurrent groups of fields, one launch per stage and group (density packing, "
                    "analysis contraction, split-K sum and patch combination, radial scans, coefficient "
                    "packing, synthesis contraction)") if launches < len(specs) else
                   "per-field solves on parallel branches",
        "graph_forms": modes,
        "graph_branches": b.branches(), "field_groups": groups,
        "analysis_splits_chosen": {str(v): splits.count(v) for v in sorted(set(splits))},
        "sum_of_solo_solves_ms": solo_ms,
        "fp64_gpu_path": {"value": len(specs) * 1e3 / ms64, "unit": "field solves/s", "ms_per_step": ms64},
        "speedup_vs_fp64": ms64 / ms,
        "fp64_ozaki": {"value": len(specs) * 1e3 / ms_oz, "unit": "field solves/s", "ms_per_step": ms_oz,
                       "speedup_vs_fp64": ms64 / ms_oz,
                       "phi_rel_max_pointwise_vs_fp64_worst_field": err_oz},
        "phi_rel_max_pointwise_vs_fp64_worst_field": err,
        "l2": "L2 flushed (252 MB write) before every timed step",
    }
    b.close()
    return res


# ---------------------------------------------------------------------------
# reference arm: the float64 oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, dist):
    """The CPU float64 oracle (the deliberately plain restatement of the
    method that the library is checked against), timed as it stands: each
    step is one full solve of the workload on every host core, unless
    (steps + warmup) full solves would not fit in --ref-budget-s; then each
    step evaluates an equal share of the cells (labelled in the line), and
    ms_per_step is still the time a step actually took."""
    if dist.rank != 0:
        return None
    import numpy as np
    from paper_1806_04593_gb300 import inputs
    gradient = not args.no_grad
    spec = inputs.production_grid()
    ry, rg = inputs.density_for(spec)
    og = oracle_grid(spec)
    if args.ref_cells_div > 1:
        div, t_full = args.ref_cells_div, None
    else:
        t0 = time.perf_counter()
        og.solve(ry, rg, gradient=gradient)             # a full solve, measured (counts as a warm-up step)
        t_full = time.perf_counter() - t0
        div = 1
        while (args.steps + args.warmup - 1) * t_full / div > args.ref_budget_s and div < 64:
            div *= 2
    cells = None if div == 1 else np.arange(0, spec.n_ang, div)
    for _ in range(max(0, args.warmup - (0 if t_full is None else 1))):
        og.solve(ry, rg, gradient=gradient, cells=cells)
    per = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        og.solve(ry, rg, gradient=gradient, cells=cells)
        per.append(time.perf_counter() - t0)
    step_s = sum(per) / len(per)
    if div == 1:
        value = 1.0 / step_s
        sample = (f"one full solve per step (all cells, Phi{' and -grad Phi' if gradient else ''}), "
                  f"numpy float64 oracle, BLAS on {os.cpu_count()} host cores, tables prebuilt")
    elif t_full is not None:
        value = 1.0 / t_full
        sample = (f"full solves would exceed {args.ref_budget_s:.0f} s: each step evaluates 1/{div} of the "
                  f"cells (ms_per_step is that step's measured time); value = the measured full warm-up solve "
                  f"({t_full:.2f} s)")
    else:
        t0 = time.perf_counter()
        for rho in (ry, rg):
            og.radial_sums(*og.analysis(rho))
        fix = time.perf_counter() - t0
        value = 1.0 / (fix + max(step_s - fix, 0.0) * div)
        sample = (f"each step evaluates 1/{div} of the cells (ms_per_step is that step's measured time); "
                  f"value extrapolated: analysis + radial sums ({fix:.2f} s) plus the evaluation time x{div}")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * step_s, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "1-degree Yin-Yang grid, 2 x 90 x 270 cells, n_r=550, l_max=25, "
                                   + ("Phi and -grad Phi" if gradient else "Phi only"),
                       "n_r": spec.n_r, "n_theta": spec.n_theta, "n_phi": spec.n_phi,
                       "l_max": spec.lmax, "gradient": gradient, "sampled_cells_div": div},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    dist = Dist(init=(args.impl == "ours"))
    try:
        out = run_reference(args, dist) if args.impl == "reference" else run_ours(args, dist)
        if out is not None and dist.rank == 0:
            print(json.dumps(out))
    finally:
        dist.close()


if __name__ == "__main__":
    main()
