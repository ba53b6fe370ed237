#!/usr/bin/env python3
"""Benchmark of the D2V16 MRT flux-limiter FDLBM step on one GB300 (or N replicas).

Workload: the 8192 x 8192 doubly periodic low-Mach shear layer (rho = T = 1,
u = +-0.05 tanh layers, seeded v perturbation; gamma = 1.4, Pr = 0.71,
dt = 1e-5), the largest grid of the benchmark set.  A step is one pass of the
hot path: ghost fill + fused collide/convect kernel; the float64 totals
reduction (rho, j, e) runs every 100 steps and once at the end.

The headline line is the FP32 deviation mode (f stored as f - f^eq0 in float32,
bound by HBM: 128 algorithmic bytes per cell-update); the FP64 mode (bound by the
float64 pipe) is measured in the same run and reported under "fp64".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(weak scaling, no collective on the data path); the timing is max over ranks.
`--impl reference` times the CPU oracle (the plain FP64 reference
implementation of the same step) on a bounded crop of the same workload.
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

METRIC = "D2V16 cell-updates/s"
UNIT = "cell-updates/s"
N_GRID = 8192
BYTES_PER_CELL = {"f32": 128, "f64": 256}     # read 16 populations + write 16 populations
# Algorithmic float64 operations per cell-update of the symmetry-factored step
# (each add, multiply, FMA or division = one float64-pipe operation; the limiter's
# magnitude comparisons and sign logic are exact integer operations and not counted).
FP64_OPS_PER_CELL = 335
TOTALS_EVERY = 100
# DRAM bytes (read + write) per cell of one fused-step launch from an ncu capture of the
# current kernels (profiles/k_step_tma_*_shear_layer.md: 4096^2 FP32, 2048^2 FP64, scaled by
# the cell count); None once the kernel changes and until it is captured again.
TRAFFIC_PER_CELL = {"f32": 125.87, "f64": 251.43}   # dram bytes per cell, ncu captures in profiles/


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=N_GRID, help="grid edge (default 8192)")
    ap.add_argument("--mode", default="both", choices=["both", "f32", "f64"],
                    help="precisions to measure (the headline line is FP32 unless --mode f64)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--step-kernel", type=int, default=0,
                    help="lbm_options.step_kernel (0 = automatic, 1/3/4/7 plain, 2 TMA tiles, 5 streaming, "
                         "6 double-buffered TMA tiles)")
    ap.add_argument("--serving-requests", type=int, default=64,
                    help="requests of the serving measurement (0 = skip)")
    ap.add_argument("--serving-steps", type=int, default=200)
    return ap.parse_args(argv)


# ------------------------------------------------------------------------- helpers
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_max(value: float, world: int, device=None) -> float:
    """Max over ranks (identity for one process)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during a timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def pinned_like(a):
    import numpy as np
    import torch
    t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
    out = t.numpy()
    np.copyto(out, a)
    return out, t


# ------------------------------------------------------------------------- GPU arm
KERNEL_NAMES = {1: "k_step<{r},{d},MC,256>", 2: "k_step_tma<{r},{d},MC>", 3: "k_step<{r},{d},MC,128>",
                4: "k_step<{r},{d},MC,512>", 5: "k_step_stream<{r},{d},MC>", 6: "k_step_tma_pipe<{r},{d},MC>",
                7: "k_step<{r},{d},MC,64>"}


def run_mode(lbm, p, precision, steps, warmup, device, world, step_kernel=0):
    """Time `steps` steps (device events) and one end-to-end pass (host buffers)."""
    import numpy as np
    import torch

    s = lbm.Solver.from_problem(p, precision=precision, device=device, step_kernel=step_kernel)
    kernel = KERNEL_NAMES[s.step_kernel].format(r="float" if precision else "double",
                                                 d="dev" if precision else "plain")
    s.init(*p.fields())
    s.step(warmup)
    totals_start = s.totals()
    torch.cuda.synchronize(device)
    stream = torch.cuda.current_stream(device)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    barrier(world)
    torch.cuda.synchronize(device)
    lbm.lbm_profile_begin(s.h, steps)
    ev0.record(stream)
    done = 0
    while done < steps:
        n = min(TOTALS_EVERY, steps - done)
        s.step(n)
        done += n
        launches += 2 * n
        s.totals()                                 # float64 reduction of rho, j, e
        launches += 2
    ev1.record(stream)
    torch.cuda.synchronize(device)
    prof = lbm.lbm_profile_end(s.h)
    barrier(world)
    ms_local = ev0.elapsed_time(ev1)
    ms = reduce_max(ms_local, world, torch.device("cuda", device))
    step_kernel_ms = prof[0] / max(prof[1], 1)
    ghost_ms = prof[2] / max(prof[3], 1)
    totals_end = s.totals()
    s.close()

    # end to end through the C interface: host fields -> init -> steps -> moments -> host
    rho, ux, uy, T = (pinned_like(a) for a in p.fields())
    outs = [pinned_like(np.zeros((p.ny, p.nx))) for _ in range(4)]
    torch.cuda.synchronize(device)
    barrier(world)
    t0 = time.perf_counter()
    s = lbm.Solver.from_problem(p, precision=precision, device=device, step_kernel=step_kernel)
    s.init(rho[0], ux[0], uy[0], T[0])
    s.step(steps)
    rc = lbm.lbm_moments(s.h, outs[0][0], outs[1][0], outs[2][0], outs[3][0], None)
    t1 = time.perf_counter()
    s.close()
    e2e_s = reduce_max(t1 - t0, world, torch.device("cuda", device))
    return {
        "ms": ms, "ms_local": ms_local, "step_kernel_ms": step_kernel_ms, "ghost_ms": ghost_ms,
        "launches": launches, "e2e_s": e2e_s, "e2e_rc": rc, "totals": [float(x) for x in totals_end],
        "kernel": kernel, "totals_drift": totals_drift(totals_start, totals_end, steps),
    }


def totals_drift(t0, t1, steps):
    """Drift of the conserved totals (mass, momentum, energy; exactly conserved by the flux
    form on a periodic grid) over `steps` steps, relative to the mass and energy totals."""
    m, e = abs(float(t0[0])), abs(float(t0[3]))
    return {"steps": steps, "mass": abs(float(t1[0]) - float(t0[0])) / m,
            "momentum_x": abs(float(t1[1]) - float(t0[1])) / m,
            "momentum_y": abs(float(t1[2]) - float(t0[2])) / m,
            "energy": abs(float(t1[3]) - float(t0[3])) / e}


def precision_compare(lbm, p, device, steps=20):
    """FP32 deviation mode against FP64 on the same fields after `steps` steps: L1 and max
    relative errors of rho, u (as a vector) and T over the whole grid."""
    import numpy as np
    out = {}
    for prec in (lbm.LBM_FP64, lbm.LBM_FP32_DEV):
        s = lbm.Solver.from_problem(p, precision=prec, device=device)
        s.init(*p.fields())
        s.step(steps)
        out[prec] = s.moments()
        s.close()
    a, b = out[lbm.LBM_FP32_DEV], out[lbm.LBM_FP64]

    def rel(x, y):
        return {"l1": float(np.abs(x - y).sum() / np.abs(y).sum()), "max": float(np.abs(x - y).max() / np.abs(y).max())}
    du = np.maximum(np.abs(a[1] - b[1]), np.abs(a[2] - b[2]))
    umax = max(np.abs(b[1]).max(), np.abs(b[2]).max())
    usum = (np.abs(b[1]) + np.abs(b[2])).sum()
    return {"steps": steps, "rho": rel(a[0], b[0]), "T": rel(a[3], b[3]),
            "u": {"l1": float(du.sum() / usum), "max": float(du.max() / umax)}}


def cpu_baseline_run(p_full, crop: int, steps_budget_s: float = 12.0, max_steps: int = 400):
    """The CPU oracle, as it stands, on a crop of the workload (all host cores)."""
    import numpy as np
    from oracle import oracle as orc
    orc.build()
    threads = os.cpu_count() or 1
    orc.set_threads(threads)
    c = min(crop, p_full.nx, p_full.ny)
    fields = [np.ascontiguousarray(a[:c, :c]) for a in p_full.fields()]
    O = orc.Oracle(c, c, p_full.dx, p_full.dt, p_full.gamma, p_full.s, p_full.limiter, p_full.bc)
    O.init(*fields)
    t0 = time.perf_counter()
    O.step(1)
    one = time.perf_counter() - t0
    n = int(max(2, min(max_steps, steps_budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    O.step(n)
    el = time.perf_counter() - t0
    O.close()
    return {"value": c * c * n / el, "unit": UNIT, "cores": orc.max_threads(), "kind": "oracle",
            "sample": f"{c}x{c} crop of the {p_full.nx}x{p_full.ny} shear layer (same dx, dt, rates), "
                      f"{n} FP64 steps, OpenMP over cells, {el:.1f} s"}


def gpu_arm(args):
    import numpy as np
    import torch
    from paper_1305_4736_gb300 import build, lbm, workloads as wl

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    device = local
    torch.cuda.set_device(device)
    if rank == 0:
        build.build()
    barrier(world)
    lbm.load()

    p = wl.shear_layer(args.n)
    cells = p.nx * p.ny
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))

    if args.mode == "f64":
        line = fp64_line(lbm, p, args, device, world, hbm)
        line["fp64_headline"] = True
        finish(line, p, args, rank, world)
        return
    with ClockSampler(device) as clk32:
        r32 = run_mode(lbm, p, lbm.LBM_FP32_DEV, args.steps, args.warmup, device, world, args.step_kernel)
    clocks = clk32.summary()
    value = world * cells * args.steps / (r32["ms"] * 1e-3)
    ach = BYTES_PER_CELL["f32"] * cells / (r32["step_kernel_ms"] * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r32["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"shear_layer_{p.nx}x{p.ny}", "mode": "FP32 deviation storage (g = f - f^eq0)",
                   "grid": [p.nx, p.ny], "cells_per_gpu": cells, "dt": p.dt, "dx": p.dx, "gamma": p.gamma,
                   "Pr": p.Pr, "limiter": "MC", "boundaries": "doubly periodic",
                   "totals_every": TOTALS_EVERY, "l2": "inputs larger than L2 (4.3 GB per population buffer)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "traffic": (TRAFFIC_PER_CELL["f32"] * cells if TRAFFIC_PER_CELL.get("f32") else None),
                     "kernel": r32["kernel"],
                     "kernel_ms": r32["step_kernel_ms"], "algorithmic_bytes_per_launch": BYTES_PER_CELL["f32"] * cells,
                     "peak_source": f"{peak_src} hbm_gbs"},
        "e2e": {"value": world * cells * args.steps / r32["e2e_s"], "unit": UNIT,
                "h2d_bytes_per_step": 4 * 8 * cells / args.steps, "d2h_bytes_per_step": 4 * 8 * cells / args.steps,
                "note": "lbm_create + lbm_init (4 float64 host fields, pinned) + steps + lbm_moments "
                        "(rho, u, v, T to host), wall clock"},
        "gpu_launches": r32["launches"],
        "clocks": clocks,
        "kernel_ms": {"step": r32["step_kernel_ms"], "ghost": r32["ghost_ms"]},
        "totals_drift": r32["totals_drift"],
    }
    if args.mode == "both":
        line["fp64"] = fp64_line(lbm, p, args, device, world, hbm)
        if rank == 0:
            line["precision"] = precision_compare(lbm, p, device)
    finish(line, p, args, rank, world)


def fp64_line(lbm, p, args, device, world, hbm):
    cells = p.nx * p.ny
    k64 = max(3, args.steps // 10) if args.mode == "both" else args.steps
    peak64 = lbm.lbm_peak_fp64(device)
    with ClockSampler(device) as clk64:
        r64 = run_mode(lbm, p, lbm.LBM_FP64, k64, args.warmup, device, world, args.step_kernel)
    ops = FP64_OPS_PER_CELL * cells / (r64["step_kernel_ms"] * 1e-3)
    peak_ops = peak64 / 2.0
    return {
        "metric": METRIC, "value": world * cells * k64 / (r64["ms"] * 1e-3), "unit": UNIT, "steps": k64,
        "warmup": args.warmup, "n_gpus": world, "ms_per_step": r64["ms"] / k64, "dtype": "f64",
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic",
        "config": {"workload": f"shear_layer_{p.nx}x{p.ny}", "mode": "FP64 (f stored in float64)",
                   "grid": [p.nx, p.ny], "l2": "inputs larger than L2 (8.6 GB per population buffer)"},
        "roofline": {"bound": "alu", "achieved": ops / 1e12, "peak": peak_ops / 1e12,
                     "unit": "T fp64-op/s", "frac": ops / peak_ops,
                     "traffic": (TRAFFIC_PER_CELL["f64"] * cells if TRAFFIC_PER_CELL.get("f64") else None),
                     "kernel": r64["kernel"], "kernel_ms": r64["step_kernel_ms"],
                     "algorithmic_ops_per_cell": FP64_OPS_PER_CELL,
                     "peak_source": "measured fp64 FMA-chain rate (lbm_peak_fp64), one op per FMA",
                     "hbm_frac": BYTES_PER_CELL["f64"] * cells / (r64["step_kernel_ms"] * 1e-3) / 1e9 / hbm},
        "e2e": {"value": world * cells * k64 / r64["e2e_s"], "unit": UNIT,
                "h2d_bytes_per_step": 4 * 8 * cells / k64, "d2h_bytes_per_step": 4 * 8 * cells / k64},
        "gpu_launches": r64["launches"], "clocks": clk64.summary(),
        "kernel_ms": {"step": r64["step_kernel_ms"], "ghost": r64["ghost_ms"]},
        "totals_drift": r64["totals_drift"],
    }


def serving_measure(count, steps, max_nx, max_ny, device, seed=1305):
    """Continuous-batching serving of a seeded mixed request stream (Riemann, Couette,
    shock-interface; FP32/FP64 50/50) against one-at-a-time FP64 solving of the same
    requests.  Arrivals are Poisson at 1.5x the measured one-at-a-time FP64 rate."""
    from paper_1305_4736_gb300 import serving, workloads as wl
    be = serving.GpuBackend(device)
    reqs = wl.serving_requests(count=count, seed=seed, rate_hz=1.0, max_nx=max_nx, max_ny=max_ny, steps=steps)
    warm = [dict(r) for r in reqs[:2]]
    serving.one_at_a_time(be, warm, precision=0)
    wall64, _ = serving.one_at_a_time(be, reqs, precision=0)
    rate64 = len(reqs) / wall64
    reqs = wl.serving_requests(count=count, seed=seed, rate_hz=1.5 * rate64, max_nx=max_nx, max_ny=max_ny,
                               steps=steps)
    res, st = serving.Engine(be, budget_bytes=64 << 30, chunk=100, realtime=True).run(reqs)
    _, cap = serving.Engine(be, budget_bytes=64 << 30, chunk=100, realtime=False).run(reqs)
    return {"capacity_solves_per_s": cap.solves_per_s, "capacity_note": "all requests available at t = 0","requests": count, "steps_per_request": steps, "grids": f"nx 64..{max_nx}, ny 4..{max_ny} log-uniform",
            "arrival_rate_hz": 1.5 * rate64, "solves_per_s": st.solves_per_s, "p50_s": st.p50, "p99_s": st.p99,
            "wall_s": st.wall, "max_resident_solves": st.max_resident_solves,
            "max_resident_gb": st.max_resident_bytes / 1e9, "cell_updates_per_s": st.cell_updates / st.wall,
            "one_at_a_time_fp64_solves_per_s": rate64, "speedup_vs_one_at_a_time_fp64": st.solves_per_s / rate64}


def batch_measure(device, steps=20, warmup=3, seed=1305):
    """Batched stepping (one lbm_batch: a ghost launch and a fused-step launch per step over a
    tile list of all grids) of 24 uneven float32 shear-layer grids whose buffers exceed L2,
    against stepping the same grids one at a time on their automatic kernels."""
    import numpy as np
    import torch
    from paper_1305_4736_gb300 import lbm, workloads as wl
    rng = np.random.default_rng(seed)
    sizes = [(int(rng.choice([512, 768, 1024, 1536, 2048])), int(rng.choice([256, 384, 512, 768, 1024])))
             for _ in range(24)]
    solvers = []
    for k, (nx, ny) in enumerate(sizes):
        p = wl.shear_layer(nx, ny=ny, seed=seed + k)
        s = lbm.Solver.from_problem(p, precision=1, device=device)
        s.init(*p.fields())
        solvers.append(s)
    cells = sum(nx * ny for nx, ny in sizes)
    stream = torch.cuda.current_stream(device)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn(warmup)
        torch.cuda.synchronize(device)
        ev0.record(stream)
        fn(steps)
        ev1.record(stream)
        torch.cuda.synchronize(device)
        return ev0.elapsed_time(ev1) / steps

    b = lbm.Batch(solvers)
    ms = timed(b.step)
    b.close()

    def solo(n):
        for s in solvers:
            s.step(n)
    ms_solo = timed(solo)
    for s in solvers:
        s.close()
    gbs = 128.0 * cells / (ms * 1e-3) / 1e9
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    return {"grids": len(sizes), "cells": cells, "sizes": "nx 512..2048, ny 256..1024 (seeded)",
            "dtype": "f32", "bytes_per_step": 128 * cells, "steps": steps, "warmup": warmup,
            "ms_per_step": ms, "cell_updates_per_s": cells / (ms * 1e-3),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "peak_source": f"{peak_src} hbm_gbs", "traffic": None,
                         "kernel": "k_ghost_batch, then each grid's k_step_tma<float,dev,MC> on 8 forked "
                                   "streams (grids under 512 cells per SM: k_step_batch), in one CUDA graph"},
            "one_at_a_time_ms_per_step": ms_solo, "speedup_vs_one_at_a_time": ms_solo / ms}


def finish(line, p, args, rank, world):
    if rank == 0 and args.serving_requests > 0:
        import torch
        line["batch"] = batch_measure(torch.cuda.current_device())
        import torch
        line["serving"] = serving_measure(args.serving_requests, args.serving_steps, 1024, 256,
                                          torch.cuda.current_device())
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_run(p, 1024)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------- reference arm
def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    from oracle import oracle as orc
    from paper_1305_4736_gb300 import workloads as wl

    orc.build()
    threads = os.cpu_count() or 1
    orc.set_threads(threads)
    p = wl.shear_layer(args.n)
    crop = min(512, p.nx)
    fields = [np.ascontiguousarray(a[:crop, :crop]) for a in p.fields()]
    O = orc.Oracle(crop, crop, p.dx, p.dt, p.gamma, p.s, p.limiter, p.bc)
    O.init(*fields)
    O.step(args.warmup)
    t0 = time.perf_counter()
    O.step(args.steps)
    el = time.perf_counter() - t0
    O.close()
    value = crop * crop * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"shear_layer_{p.nx}x{p.ny}", "grid": [p.nx, p.ny],
                   "sample": f"{crop}x{crop} crop per step", "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc.max_threads(), "kind": "oracle",
                         "sample": f"{crop}x{crop} crop of the {p.nx}x{p.ny} shear layer, "
                                   f"{args.warmup}+{args.steps} FP64 steps, OpenMP over cells"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
