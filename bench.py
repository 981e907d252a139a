#!/usr/bin/env python3
"""Benchmark of the Yin-Yang multipole gravity solver on GB300.

Workload: the 1-degree Yin-Yang grid (90 x 270 cells per patch), 550
log-spaced zones in [1e-4, 1], l_max = 25, with the seeded proto-neutron-star
density; tables prebuilt.  One step = one solve of Phi and -grad Phi on both
patches (analysis, radial scans, four synthesis contractions).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec P] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is solves/s over all ranks from
device-side CUDA events; `e2e` is the same metric through the host-buffer
entry points (pinned host buffers, host<->device copies inside the timed
region): yy_potential_host_async, whose calls overlap one solve's copy out
with the next one's copy in and solve, and, beside it, the synchronous
yy_potential_host.  The `batched` object times the 64-field workload as one
CUDA graph per step.  With several
GPUs every rank solves its own field (replicas, weak scaling).  The reference
arm times the CPU float64 oracle on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import json
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
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12     # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz


# DRAM bytes (read + write) of one synthesis launch, from an ncu capture of
# this workload (profiles/k_tc_pair_fp16x2_production.md); valid only for the
# kernel source it was taken with, null otherwise.
_TRAFFIC = {("fp16x2", True): (288.576512e6 + 798.440192e6,
                               "933feec6e70168707e470471a68dd3cfee2a75552822e0b5b580f626169b9a4c")}


def _recorded_traffic(prec, gradient):
    import hashlib
    rec = _TRAFFIC.get((prec, gradient))
    if rec is None:
        return None
    path = os.path.join(ROOT, "paper_1806_04593_gb300", "csrc", "yy_tc_pair.cuh")
    try:
        with open(path, "rb") as fh:
            digest = hashlib.sha256(fh.read()).hexdigest()
    except OSError:
        return None
    return rec[0] if digest == rec[1] else None


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "source": "fallback"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="auto")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-path", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-field batched workload")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--cpu-sample", type=int, default=4, help="oracle evaluates 1/S of the cells")
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
# the oracle on a bounded sample (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample_solve(og, ry, rg, cells, gradient):
    t0 = time.perf_counter()
    res = og.solve(ry, rg, gradient=gradient, cells=cells)
    return res, time.perf_counter() - t0


def oracle_fixed_cost(og, ry, rg):
    """Time of the density-dependent part that does not scale with the
    number of target cells (analysis and radial sums of both patches)."""
    t0 = time.perf_counter()
    for rho in (ry, rg):
        og.radial_sums(*og.analysis(rho))
    return time.perf_counter() - t0


def cpu_baseline(spec, ry, rg, gradient, sample_div):
    import numpy as np
    from oracle import OracleGrid
    og = OracleGrid(spec.r_edges, spec.n_theta, spec.n_phi, spec.delta_theta, spec.delta_phi,
                    spec.lmax, spec.G)
    cells = np.arange(0, spec.n_ang, sample_div)
    fixed = oracle_fixed_cost(og, ry, rg)
    res, t_sample = oracle_sample_solve(og, ry, rg, cells, gradient)
    t_full = fixed + (t_sample - fixed) * (spec.n_ang / cells.size)
    info = {"value": 1.0 / t_full, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"numpy float64 oracle: analysis + radial sums of both patches in full "
                       f"({fixed:.2f} s), Phi{' and -grad Phi' if gradient else ''} at 1/{sample_div} "
                       f"of the target cells ({cells.size} cells x {spec.n_r} radii, "
                       f"{t_sample - fixed:.2f} s), evaluation time scaled x{spec.n_ang / cells.size:.1f}; "
                       f"tables prebuilt; numpy BLAS threading")}
    return info, res, cells


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

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

    spec = inputs.production_grid()
    grid = yy.Grid.from_spec(spec)
    prec = args.prec
    if prec == "auto":
        prec = "fp16x2"
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

    def solve():
        grid.potential(ry, rg, phi_y, phi_g, g_y, g_g, prec=prec, stream=stream)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    launches = yy.yy_last_launch_count(grid.handle)

    # ---- device-timed region: the host enqueues every step without waiting
    # (as a caller's time loop would), so the events see device time only
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(dist.local)
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    w0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()                              # evict L2 between steps (outside the events)
        starts[i].record(stream)
        solve()
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    dist.barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]

    # ---- stage breakdown (the library's CUDA events between the stages, read
    # back after every step), on a separate pass of the same steps
    prof_steps = min(args.steps, 50)
    stage_tot = {k: 0.0 for k in yy.STAGES}
    yy.yy_grid_set_profiling(grid.handle, 1)
    for i in range(prof_steps):
        flush.zero_()
        solve()
        st, stages = yy.yy_grid_stage_ms(grid.handle)
        for k in stage_tot:
            stage_tot[k] += stages[k]
    yy.yy_grid_set_profiling(grid.handle, 0)
    torch.cuda.synchronize()
    dev_s = sum(step_ms) / 1e3
    dev_s_max = dist.max(dev_s)
    value = dist.world * args.steps / dev_s_max

    # ---- end to end through the host-buffer entry point
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_ry, h_rg = pin(ry_np), pin(rg_np)
    h_py = torch.empty(shape, dtype=torch.float64).pin_memory()
    h_pg = torch.empty(shape, dtype=torch.float64).pin_memory()
    h_gy = torch.empty((3,) + shape, dtype=torch.float64).pin_memory() if gradient else None
    h_gg = torch.empty((3,) + shape, dtype=torch.float64).pin_memory() if gradient else None
    pcode = yy.PRECISIONS[prec]
    for _ in range(max(1, args.warmup // 2)):
        yy.yy_potential_host(grid.handle, h_ry, h_rg, h_py, h_pg, h_gy, h_gg, pcode, stream)
    e2e_steps = min(args.steps, 50)
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        st = yy.yy_potential_host(grid.handle, h_ry, h_rg, h_py, h_pg, h_gy, h_gg, pcode, stream)
        assert st == yy.YY_OK, yy.yy_status_string(st)
    e2e_sync_s = dist.max(time.perf_counter() - t0) / e2e_steps
    # the pipelined entry point: two host output sets in turn, each call's
    # copy out overlapping the next call's copy in and solve
    h_out = [(h_py, h_pg, h_gy, h_gg),
             tuple(torch.empty_like(x).pin_memory() if x is not None else None for x in (h_py, h_pg, h_gy, h_gg))]
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

    # ---- roofline of the dominant kernel: the synthesis stage (one launch of
    # k_tc_pair for all contractions on the tensor-core forms; one k_gemm_tn
    # launch per contraction on the CUDA-core forms), timed by the library's
    # CUDA events on the solve's stream
    n_synth = 4 if gradient else 1
    synth_ms = stage_tot["synthesis"] / prof_steps
    synth_flop = n_synth * 2.0 * (2 * spec.n_r) * grid.n_lm * spec.n_ang   # 2 M N K, K = n_lm
    total_flop = grid.flops(gradient)
    products = {"fp16x2": 3, "bf16x3": 6, "tf32": 1, "fp64": 1, "fp32": 1, "fp64_ozaki": 26}[prec]
    pieces_bytes = {"fp16x2": 4, "bf16x3": 6, "tf32": 4, "fp64": 8, "fp32": 4, "fp64_ozaki": 12}[prec]
    cells_pad = -(-spec.n_ang // 256) * 256
    k_pad = -(-grid.n_lm // 64) * 64
    synth_bytes = (n_synth * 2 * spec.n_r * spec.n_ang * 8                  # float64 outputs
                   + n_synth * cells_pad * k_pad * pieces_bytes)             # one table pass per contraction
    peaks = _measured_peaks()
    if prec == "fp64_ozaki":
        # separable synthesis: float64 polar stage, then the azimuthal stage as
        # 26 digit products over rows (shell, j) x longitudes, K = 64
        g_rows = 2 * spec.n_r * spec.n_theta
        digit_flop = products * n_synth * 2.0 * g_rows * spec.n_phi * 64
        synth_bytes = (n_synth * 2 * spec.n_r * spec.n_ang * 8            # float64 outputs
                       + 2 * n_synth * g_rows * 64 * pieces_bytes)          # digit rows written, then read
        roof = {"bound": "tensor",
                "kernel": ("k_tc_pair<FormOzaki, 3> (azimuthal synthesis stage, digit products on tcgen05), "
                           "timed together with the float64 polar stage k_theta_ozaki"),
                "achieved": digit_flop / (synth_ms / 1e3) / 1e12, "peak": peaks["bf16_tflops"],
                "unit": "TFLOP/s", "traffic": None,
                "flops_counted": (f"hardware: {products} bf16 digit products x 2 M N K, M = 2 n_r n_theta, "
                                  f"N = n_phi, K = 64, {n_synth} field(s)"),
                "peak_source": "measured bf16 burst (MEASURED_PEAKS.json)"}
    elif prec in ("fp64", "fp32"):
        # the CUDA-core forms synthesise in separable form by default: a polar
        # stage (K = n_lm per theta row) and an azimuthal one (K = 2 l_max + 1)
        g_rows = 2 * spec.n_r * spec.n_theta
        sep_flop = n_synth * (2.0 * g_rows * grid.n_lm + 2.0 * g_rows * spec.n_phi * (2 * spec.lmax + 1))
        t = "double" if prec == "fp64" else "float"
        roof = {"bound": "alu", "kernel": f"k_sep_synth<{t}> (separable synthesis, CUDA cores)",
                "achieved": sep_flop / (synth_ms / 1e3) / 1e12, "unit": "TFLOP/s", "traffic": None,
                "flops_counted": "2 x (theta-stage + phi-stage multiply-adds) of the separable synthesis"}
        if prec == "fp64":
            roof.update(peak=FP64_PEAK_TFLOPS, peak_source="derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz")
        else:
            roof.update(peak=152 * 128 * 2 * 2.070e9 / 1e12,
                        peak_source="derived: 152 SMs x 128 FFMA/clk x 2 flop x 2070 MHz")
    else:
        ratio = 0.5 if prec == "tf32" else 1.0
        roof = {"bound": "tensor", "kernel": f"k_tc_pair<{prec}> (synthesis, tcgen05 cta_group::2)",
                "achieved": products * synth_flop / (synth_ms / 1e3) / 1e12,
                "peak": peaks["bf16_tflops"] * ratio, "unit": "TFLOP/s",
                "traffic": _recorded_traffic(prec, gradient),
                "flops_counted": (f"hardware: {products} tensor-core products x 2MNK, K = n_lm, "
                                  f"{n_synth} contraction(s) in one launch"),
                "peak_source": ("measured bf16 burst (MEASURED_PEAKS.json)"
                                + (" x 0.5 (tf32 nominal ratio)" if prec == "tf32" else ""))}
    roof["hbm"] = {"algorithmic_bytes": synth_bytes,
                   "achieved_gbs": synth_bytes / (synth_ms / 1e3) / 1e9,
                   "peak_gbs": peaks["hbm_gbs"],
                   "frac": synth_bytes / (synth_ms / 1e3) / 1e9 / peaks["hbm_gbs"]}
    roof["frac"] = roof["achieved"] / roof["peak"]

    # ---- the plain float64 GPU path on the same grid, for comparison
    fp64_path = None
    if prec != "fp64" and not args.no_fp64_path:
        grid.potential(ry, rg, phi_y, phi_g, g_y, g_g, prec="fp64", stream=stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(2):
            grid.potential(ry, rg, phi_y, phi_g, g_y, g_g, prec="fp64", stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / 2
        fp64_path = {"value": 1e3 / ms64, "unit": UNIT, "ms_per_step": ms64,
                     "headline_speedup": value / dist.world / (1e3 / ms64)}
        # the same float64 accuracy with the synthesis's azimuthal stage on the
        # tensor cores (Ozaki scheme), and its largest difference from the
        # CUDA-core float64 result
        try:
            grid.prepare("fp64_ozaki")
        except yy.YYError as exc:
            fp64_path["ozaki"] = {"unavailable": str(exc)}
        else:
            if prec == "fp64_ozaki":
                fp64_path["ozaki"] = {"same_as": "the headline value of this line"}
            else:
                ref64 = {"phi_yin": phi_y.clone(), "phi_yang": phi_g.clone()}
                if gradient:
                    ref64["grad_yin"], ref64["grad_yang"] = g_y.clone(), g_g.clone()
                grid.potential(ry, rg, phi_y, phi_g, g_y, g_g, prec="fp64_ozaki", stream=stream)
                torch.cuda.synchronize()
                got = {"phi_yin": phi_y, "phi_yang": phi_g, "grad_yin": g_y, "grad_yang": g_g}
                diff = max(float((got[k] - v).abs().max() / v.abs().max()) for k, v in ref64.items())
                e0.record(stream)
                for _ in range(3):
                    grid.potential(ry, rg, phi_y, phi_g, g_y, g_g, prec="fp64_ozaki", stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                msoz = e0.elapsed_time(e1) / 3
                fp64_path["ozaki"] = {"value": 1e3 / msoz, "unit": UNIT, "ms_per_step": msoz,
                                      "speedup_vs_fp64_path": ms64 / msoz,
                                      "rel_max_diff_vs_fp64_path": diff,
                                      "precision": "fp64_ozaki (float64 results; the azimuthal stages of "
                                                   "analysis and synthesis as balanced 8-bit digit "
                                                   "products on tcgen05, exact per level)"}
        solve()                                   # leave the headline form's result in place
        torch.cuda.synchronize()

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dev_s_max * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32", "fp16x2": "fp16x2 (fp32 accumulate, f64 scans)",
                  "bf16x3": "bf16x3 (fp32 accumulate, f64 scans)",
                  "tf32": "tf32 (fp32 accumulate, f64 scans)",
                  "fp64_ozaki": "f64 (Ozaki: azimuthal stages as 8-bit digit products on tcgen05, exact per level)"}[prec],
        "data": "synthetic (seeded proto-neutron-star density, l<=4 angular perturbation)",
        "config": {"workload": "1-degree Yin-Yang grid, 2 x 90 x 270 cells, n_r=550 log r in [1e-4,1], "
                               "l_max=25, Phi and -grad Phi per solve" if gradient else
                               "1-degree Yin-Yang grid, 2 x 90 x 270 cells, n_r=550, l_max=25, Phi only",
                   "n_r": spec.n_r, "n_theta": spec.n_theta, "n_phi": spec.n_phi, "l_max": spec.lmax,
                   "gradient": gradient, "precision": prec, "parallelism": f"replicas x{dist.world}",
                   "l2": "L2 flushed (256 MB write) before every timed step"},
        "gemm_tflops": total_flop / (dev_s_max / args.steps) / 1e12,
        "gemm_tflops_hardware": products * total_flop / (dev_s_max / args.steps) / 1e12,
        "fp64_gpu_path": fp64_path,
        "stage_ms": {k: v / prof_steps for k, v in stage_tot.items()},
        "stage_ms_steps": prof_steps,
        "wall_s": wall,
        "roofline": roof,
        "e2e": {"value": dist.world / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "api": "yy_potential_host_async (pinned host buffers, copies overlapped across calls), "
                       f"{e2e_steps} calls then yy_potential_host_wait",
                "synchronous_call": {"value": dist.world / e2e_sync_s, "unit": UNIT,
                                     "api": "yy_potential_host (copy in, solve, copy out, sync per call)"}},
        "gpu_launches": launches * args.steps,
        "clocks": clk,
    }

    # ---- the batched workload (uneven fields in one graph), rank-local
    if not args.no_batch:
        out["batched"] = run_batched(args, prec, gradient, dev, stream, flush)

    # ---- CPU baseline (oracle) and error vs the float64 oracle, rank 0 at N=1
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        info, ref, cells = cpu_baseline(spec, ry_np, rg_np, gradient, args.cpu_sample)
        out["cpu_baseline"] = info
        j, k = np.divmod(cells, spec.n_phi)
        err = {}
        got = {"phi_yin": phi_y, "phi_yang": phi_g, "grad_yin": g_y, "grad_yang": g_g}
        for key in ("phi_yin", "phi_yang") + (("grad_yin", "grad_yang") if gradient else ()):
            a = got[key].cpu().numpy()
            a = a[:, j, k] if key.startswith("phi") else a[:, :, j, k]
            r = ref[key]
            err[key] = {"rel_max": float(np.abs(a - r).max() / np.abs(r).max()),
                        "rel_l2": float(np.linalg.norm(a - r) / np.linalg.norm(r))}
        out["error_vs_fp64_oracle"] = err
    grid.close()
    return out


def run_batched(args, prec, gradient, dev, stream, flush):
    """The batched workload: 64 fields of uneven size (n_r ~ U{100..600}, 2 /
    1.5 / 1 degree cells, l_max ~ U{10..40}), the analysis of each field picked
    by yy_batch_tune, all solves replayed as one CUDA graph per step.  Reports
    field solves/s in the given form and in float64 on the same batch, and the
    error of Phi against the float64 batch field by field."""
    import torch

    from paper_1806_04593_gb300 import inputs, yy

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
        for _ in range(warmup):
            step(form)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            step(form)
            e1.record(stream)
        torch.cuda.synchronize()
        st = b.device_status()
        assert st == yy.YY_OK, yy.yy_status_string(st)
        return sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps

    ms = timed(prec, args.batch_steps, max(3, args.warmup))
    launches = b.launch_count()
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
    ms64 = timed("fp64", 2, 1)
    err = 0.0
    for (py, pg), o in zip(phi, outs):
        for got, ref in ((py, o[0]), (pg, o[1])):
            err = max(err, float((got - ref).abs().max() / ref.abs().max()))
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
        "graph_branches": b.branches(),
        "analysis_splits_chosen": {str(v): splits.count(v) for v in sorted(set(splits))},
        "sum_of_solo_solves_ms": solo_ms,
        "fp64_gpu_path": {"value": len(specs) * 1e3 / ms64, "unit": "field solves/s", "ms_per_step": ms64},
        "speedup_vs_fp64": ms64 / ms,
        "phi_rel_max_vs_fp64_worst_field": err,
        "l2": "L2 flushed (256 MB write) before every timed step",
    }
    b.close()
    return res


def run_reference(args, dist):
    """CPU float64 oracle on a bounded sample of the same workload."""
    if dist.rank != 0:
        return None
    from oracle import OracleGrid
    import numpy as np
    from paper_1806_04593_gb300 import inputs
    gradient = not args.no_grad
    spec = inputs.production_grid()
    ry, rg = inputs.density_for(spec)
    og = OracleGrid(spec.r_edges, spec.n_theta, spec.n_phi, spec.delta_theta, spec.delta_phi,
                    spec.lmax, spec.G)
    # bounded sample: the whole run stays near a minute of CPU time (about 1.1 s
    # per step at 1/4 of the cells), so long runs evaluate fewer cells per step
    div = max(args.cpu_sample, -(-4 * (args.steps + args.warmup) // 60))
    cells = np.arange(0, spec.n_ang, div)
    scale = spec.n_ang / cells.size
    for _ in range(args.warmup):
        oracle_sample_solve(og, ry, rg, cells, gradient)
    per = []
    for _ in range(args.steps):
        fixed = oracle_fixed_cost(og, ry, rg)
        _, t = oracle_sample_solve(og, ry, rg, cells, gradient)
        per.append(fixed + (t - fixed) * scale)
    value = args.steps / sum(per)
    sample = (f"float64 oracle; per step: analysis + radial sums of both patches in full, "
              f"Phi{' and -grad Phi' if gradient else ''} at 1/{div} of the cells, "
              f"evaluation time scaled x{scale:.1f}")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "1-degree Yin-Yang grid, 2 x 90 x 270 cells, n_r=550, l_max=25, "
                                   + ("Phi and -grad Phi" if gradient else "Phi only"),
                       "n_r": spec.n_r, "n_theta": spec.n_theta, "n_phi": spec.n_phi,
                       "l_max": spec.lmax, "gradient": gradient},
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
