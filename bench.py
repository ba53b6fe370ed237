#!/usr/bin/env python3
"""Benchmark of the D2V16 MRT flux-limiter FDLBM step on one GB300 (or N replicas).

Workload: the 8192 x 8192 doubly periodic low-Mach shear layer (rho = T = 1,
u = +-0.05 tanh layers, seeded v perturbation; gamma = 1.4, Pr = 0.71,
dt = 5.09e-6, a largest Courant number of 1/4), the largest grid of the benchmark set.  A step is one pass of the
hot path: ghost fill + fused collide/convect kernel; the float64 totals
reduction (rho, j, e) runs every 100 steps and once at the end.

The headline line is the FP32 deviation mode (f stored as f - f^eq0 in float32,
bound by HBM: 128 algorithmic bytes per cell-update); the FP64 mode (bound by the
float64 pipe) is measured in the same run and reported under "fp64".  The same
line carries:
  configs    every configuration of the benchmark set: the Sod tube 200x4 (a full
             2000-step solve), thermal Couette 4x200 at Pr 0.5, 1, 2, the
             shock-interface 4096x1024 in FP64 and FP32 with rooflines, and the
             oracle on all host cores and on one thread for each;
  precision  FP32 against FP64 at each stated length: the shear layer after 2000
             steps (whole field, totals drift) and the shock-interface over 5000
             steps (rho, u, T every 100 steps, Delta every 500);
  batch      24 uneven grids stepped as one batch;
  serving    the 512-request mixed stream (grids up to 2048x512, 1000 steps each),
             with FP64-only batched serving against one-at-a-time FP64.

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
# DRAM bytes (read + write) per cell of one fused-step launch from an ncu capture (profiles/:
# 4096^2 FP32, 2048^2 FP64, scaled by the cell count), each with the SHA-256 (first 16 hex digits)
# of the kernel sources it was captured from.  bench reports the traffic only while the sources
# still hash to that value, else null.
TRAFFIC_PER_CELL = {
    "f32": {"bytes": 125.89, "sources": ("lbm_step_tma.cu", "lbm_device.cuh", "lbm_tma_util.cuh"),
            "sha": "07a62d28b685263d"},
    "f64": {"bytes": 251.63, "sources": ("lbm_step_stream.cu", "lbm_device.cuh", "lbm_tma_util.cuh"),
            "sha": "01bf052590e27491"},
    "dd": {"bytes": 247.87, "sources": ("lbm_step_dd.cu", "lbm_dd.cuh", "lbm_device.cuh", "lbm_tma_util.cuh"),
           "sha": "a502465f89b98477"},
}
# float32-pipe operations (add, multiply, FMA: one each) per cell of one launch of the double-float
# float64 kernel on 32 x 32 tiles, counted by ncu on the same sources
# (profiles/k_step_dd_f64_shear_layer.md); None when the sources changed since.
DD_FP32_OPS = {"ops": 3649.3, "sha": "a502465f89b98477"}
FP32_LANES_PER_SM = 128           # float32 FMA lanes per SM per cycle (GB300)


def kernel_sources_sha(names) -> str:
    import hashlib
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_1305_4736_gb300", "csrc", n), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_launch(mode: str, cells: int, kernel: str):
    """ncu DRAM bytes of one fused-step launch scaled to `cells`, or None when the captured
    kernel is not the one that ran or its sources changed since the capture."""
    t = TRAFFIC_PER_CELL.get(mode)
    want = {"f32": "k_step_tma<", "f64": "k_step_stream<", "dd": "k_step_dd<MC>"}[mode]
    if not t or not t["bytes"] or not kernel.startswith(want) or kernel_sources_sha(t["sources"]) != t["sha"]:
        return None
    return t["bytes"] * cells


def dd_fp32_ops_per_cell():
    """ncu's float32-pipe operations per cell of the double-float kernel, while its sources
    still hash to the captured value."""
    if not DD_FP32_OPS["ops"] or kernel_sources_sha(TRAFFIC_PER_CELL["dd"]["sources"]) != DD_FP32_OPS["sha"]:
        return None
    return DD_FP32_OPS["ops"]


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
                         "6 double-buffered TMA tiles, 8/9 double-float 32x32/32x4 tiles)")
    ap.add_argument("--serving-requests", type=int, default=512,
                    help="requests of the serving measurement (0 = skip)")
    ap.add_argument("--serving-steps", type=int, default=1000)
    ap.add_argument("--serving-max-grid", type=int, nargs=2, default=(2048, 512), metavar=("NX", "NY"))
    ap.add_argument("--no-configs", action="store_true", help="skip the per-configuration measurements")
    ap.add_argument("--no-batch", action="store_true", help="skip the 24-grid batched-stepping measurement")
    ap.add_argument("--no-precision-study", action="store_true",
                    help="skip the FP32-vs-FP64 runs at each configuration's stated length")
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
                7: "k_step<{r},{d},MC,64>", 8: "k_step_dd<MC>", 9: "k_step_dd<MC,32x4>"}


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
                     "traffic": traffic_per_launch("f32", cells, r32["kernel"]),
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
    finish(line, p, args, rank, world)


def fp64_line(lbm, p, args, device, world, hbm):
    cells = p.nx * p.ny
    k64 = max(20, args.steps // 10) if args.mode == "both" else args.steps
    peak64 = lbm.lbm_peak_fp64(device)
    with ClockSampler(device) as clk64:
        r64 = run_mode(lbm, p, lbm.LBM_FP64, k64, args.warmup, device, world, args.step_kernel)
    ops = FP64_OPS_PER_CELL * cells / (r64["step_kernel_ms"] * 1e-3)
    peak_ops = peak64 / 2.0
    hbm_frac = BYTES_PER_CELL["f64"] * cells / (r64["step_kernel_ms"] * 1e-3) / 1e9 / hbm
    clocks = clk64.summary()
    if r64["kernel"].startswith("k_step_dd"):
        # double-float arithmetic on the float32 pipe: its peak from the unit counts and the
        # sampled SM clock, the executed float32 operations per cell from ncu
        import torch
        sms = torch.cuda.get_device_properties(device).multi_processor_count
        mhz = clocks.get("sm_mhz") or 2070.0
        peak32 = sms * FP32_LANES_PER_SM * mhz * 1e6
        per_cell = dd_fp32_ops_per_cell() if r64["kernel"] == KERNEL_NAMES[8] else None
        ach = per_cell * cells / (r64["step_kernel_ms"] * 1e-3) if per_cell else None
        roof = {"bound": "alu", "achieved": ach / 1e12 if ach else None, "peak": peak32 / 1e12,
                "unit": "T fp32-op/s", "frac": ach / peak32 if ach else None,
                "traffic": traffic_per_launch("dd", cells, r64["kernel"]),
                "kernel": r64["kernel"], "kernel_ms": r64["step_kernel_ms"],
                "fp32_ops_per_cell": per_cell,
                "fp32_ops_source": "ncu float32 add + multiply + FMA thread instructions per cell of this kernel",
                "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} float32 lanes x sampled SM clock {mhz:.0f} MHz",
                "fp64_pipe_equivalent": {"algorithmic_fp64_ops_per_cell": FP64_OPS_PER_CELL,
                                         "achieved": ops / 1e12, "fp64_fma_chain_rate": peak_ops / 1e12,
                                         "ratio": ops / peak_ops},
                "hbm_frac": hbm_frac}
    else:
        roof = {"bound": "alu", "achieved": ops / 1e12, "peak": peak_ops / 1e12,
                "unit": "T fp64-op/s", "frac": ops / peak_ops,
                "traffic": traffic_per_launch("f64", cells, r64["kernel"]),
                "kernel": r64["kernel"], "kernel_ms": r64["step_kernel_ms"],
                "algorithmic_ops_per_cell": FP64_OPS_PER_CELL,
                "peak_source": "measured fp64 FMA-chain rate (lbm_peak_fp64), one op per FMA",
                "hbm_frac": hbm_frac}
    return {
        "metric": METRIC, "value": world * cells * k64 / (r64["ms"] * 1e-3), "unit": UNIT, "steps": k64,
        "warmup": args.warmup, "n_gpus": world, "ms_per_step": r64["ms"] / k64,
        "dtype": "df64" if r64["kernel"].startswith("k_step_dd") else "f64",
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic",
        "config": {"workload": f"shear_layer_{p.nx}x{p.ny}", "mode": "FP64 (f stored in float64)",
                   "arithmetic": ("double-float (pairs of float32) on the float32 pipe"
                                  if r64["kernel"].startswith("k_step_dd") else "float64"),
                   "grid": [p.nx, p.ny], "l2": "inputs larger than L2 (8.6 GB per population buffer)"},
        "roofline": roof,
        "e2e": {"value": world * cells * k64 / r64["e2e_s"], "unit": UNIT,
                "h2d_bytes_per_step": 4 * 8 * cells / k64, "d2h_bytes_per_step": 4 * 8 * cells / k64},
        "gpu_launches": r64["launches"], "clocks": clocks,
        "kernel_ms": {"step": r64["step_kernel_ms"], "ghost": r64["ghost_ms"]},
        "totals_drift": r64["totals_drift"],
    }


def serving_measure(count, steps, max_nx, max_ny, device, seed=1305):
    """Continuous-batching serving of the seeded mixed request stream (Riemann, Couette,
    shock-interface; FP32/FP64 50/50; grids 64..max_nx x 4..max_ny log-uniform), and the
    comparison at equal accuracy: the same requests all in FP64, served batched (all available at
    t = 0) against one at a time.  The mixed stream is also served with Poisson arrivals at 1.5x
    the one-at-a-time FP64 rate, for time to result (p50/p99 per precision)."""
    import numpy as np
    from paper_1305_4736_gb300 import serving, workloads as wl
    be = serving.GpuBackend(device)
    reqs = wl.serving_requests(count=count, seed=seed, rate_hz=1.0, max_nx=max_nx, max_ny=max_ny, steps=steps)
    warm = [dict(r) for r in reqs[:3]]
    serving.one_at_a_time(be, warm, precision=0)
    serving.Engine(be, budget_bytes=64 << 30, chunk=100, realtime=False).run(warm)
    t0 = time.perf_counter()
    wall64, _ = serving.one_at_a_time(be, reqs, precision=0)
    rate64 = len(reqs) / wall64
    all64 = [dict(r, precision=0) for r in reqs]
    _, cap64 = serving.Engine(be, budget_bytes=64 << 30, chunk=100, realtime=False).run(all64)
    _, cap = serving.Engine(be, budget_bytes=64 << 30, chunk=100, realtime=False).run(reqs)
    reqs = wl.serving_requests(count=count, seed=seed, rate_hz=1.5 * rate64, max_nx=max_nx, max_ny=max_ny,
                               steps=steps)
    res, st = serving.Engine(be, budget_bytes=64 << 30, chunk=100, realtime=True).run(reqs)
    per = {}
    for name, prec in (("fp64", 0), ("fp32", 1)):
        lat = np.array([r.latency for r in res if r.precision == prec])
        if lat.size:
            per[name] = {"solves": int(lat.size), "p50_s": float(np.percentile(lat, 50)),
                         "p99_s": float(np.percentile(lat, 99))}
    cells = sum(r["problem"].cells for r in reqs)
    return {"requests": count, "steps_per_request": steps, "cells_total": cells,
            "grids": f"nx 64..{max_nx}, ny 4..{max_ny} log-uniform", "precisions": "FP32/FP64 50/50",
            "fp64_equal_accuracy": {
                "batched_solves_per_s": cap64.solves_per_s, "one_at_a_time_solves_per_s": rate64,
                "speedup": cap64.solves_per_s / rate64,
                "note": "every request in FP64, all available at t = 0; batched = continuous batching "
                        "through lbm_batch, one at a time = each solve alone on its automatic kernel"},
            "capacity_mixed_solves_per_s": cap.solves_per_s,
            "arrival_rate_hz": 1.5 * rate64, "solves_per_s": st.solves_per_s, "p50_s": st.p50, "p99_s": st.p99,
            "per_precision": per, "wall_s": st.wall, "max_resident_solves": st.max_resident_solves,
            "max_resident_gb": st.max_resident_bytes / 1e9, "cell_updates_per_s": st.cell_updates / st.wall,
            "seconds": time.perf_counter() - t0}


def batch_measure(device, steps=20, warmup=3, seed=1305):
    """Batched stepping (one lbm_batch: a ghost launch and one batched tile-kernel launch per
    step over the tiles of all grids) of 24 uneven float32 shear-layer grids whose buffers
    exceed L2, against stepping the same grids one at a time on their automatic kernels."""
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
                         "kernel": "k_ghost_batch, then k_step_tma_batch<MC> over the tiles of all 24 grids "
                                   "(one CTA per 32 x 16 tile), in one CUDA graph"},
            "one_at_a_time_ms_per_step": ms_solo, "speedup_vs_one_at_a_time": ms_solo / ms}


def _pinned_fields(ny, nx, count):
    import numpy as np
    return [pinned_like(np.zeros((ny, nx))) for _ in range(count)]


def timed_steps(lbm, s, steps, device):
    """Device time of `steps` steps of one context (CUDA events on its stream, no per-step
    instrumentation: on a small grid the library's per-launch events add about 9 us a step),
    then the mean duration of its fused-step and ghost launches over `steps` more steps timed
    with the library's own events."""
    import torch
    stream = torch.cuda.current_stream(device)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    ev0.record(stream)
    s.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize(device)
    ms = ev0.elapsed_time(ev1)
    lbm.lbm_profile_begin(s.h, steps)
    s.step(steps)
    torch.cuda.synchronize(device)
    prof = lbm.lbm_profile_end(s.h)
    return ms, prof[0] / max(prof[1], 1), prof[2] / max(prof[3], 1)


def kernel_name(s, precision):
    return KERNEL_NAMES[s.step_kernel].format(r="float" if precision else "double",
                                              d="dev" if precision else "plain")


def config_gpu(lbm, p, precision, steps, warmup, device, hbm, peak_ops=None):
    """Throughput of one configuration in one precision: steps timed on the device after warm-up,
    with the fused-step kernel's roofline (FP32: HBM bytes; FP64: float64 operations)."""
    s = lbm.Solver.from_problem(p, precision=precision, device=device)
    s.init(*p.fields())
    s.step(warmup)
    ms, k_ms, g_ms = timed_steps(lbm, s, steps, device)
    kern = kernel_name(s, precision)
    s.close()
    cells = p.nx * p.ny
    out = {"steps": steps, "ms_per_step": ms / steps, "us_per_step": 1e3 * ms / steps,
           "cell_updates_per_s": cells * steps / (ms * 1e-3), "kernel": kern,
           "kernel_ms": k_ms, "ghost_ms": g_ms}
    if precision:
        ach = BYTES_PER_CELL["f32"] * cells / (k_ms * 1e-3) / 1e9
        out["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                           "peak_source": f"{measured_peaks()[1]} hbm_gbs"}
    elif peak_ops:
        ops = FP64_OPS_PER_CELL * cells / (k_ms * 1e-3)
        hbm_frac = BYTES_PER_CELL["f64"] * cells / (k_ms * 1e-3) / 1e9 / hbm
        if kern.startswith("k_step_dd"):
            import torch
            sms = torch.cuda.get_device_properties(device).multi_processor_count
            peak32 = sms * FP32_LANES_PER_SM * 2070.0 * 1e6
            per_cell = dd_fp32_ops_per_cell() if kern == KERNEL_NAMES[8] else None
            ach = per_cell * cells / (k_ms * 1e-3) if per_cell else None
            out["roofline"] = {"bound": "alu", "achieved": ach / 1e12 if ach else None, "peak": peak32 / 1e12,
                               "unit": "T fp32-op/s", "frac": ach / peak32 if ach else None,
                               "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} float32 lanes x 2070 MHz",
                               "fp64_pipe_equivalent_ratio": ops / peak_ops, "hbm_frac": hbm_frac}
        else:
            out["roofline"] = {"bound": "alu", "achieved": ops / 1e12, "peak": peak_ops / 1e12,
                               "unit": "T fp64-op/s", "frac": ops / peak_ops,
                               "peak_source": "measured fp64 FMA-chain rate (lbm_peak_fp64)", "hbm_frac": hbm_frac}
    return out


def oracle_rate(p, steps, threads, crop=None):
    """The CPU oracle, as it stands, on problem p (or its leading crop x crop block): cell-updates/s."""
    import numpy as np
    from oracle import oracle as orc
    orc.build()
    orc.set_threads(threads)
    nx, ny = (p.nx, p.ny) if crop is None else (min(crop[0], p.nx), min(crop[1], p.ny))
    fields = [np.ascontiguousarray(a[:ny, :nx]) for a in p.fields()]
    O = orc.Oracle(nx, ny, p.dx, p.dt, p.gamma, p.s, p.limiter, p.bc, dy=p.dy)
    O.init(*fields)
    O.step(1)
    t0 = time.perf_counter()
    O.step(steps)
    el = time.perf_counter() - t0
    O.close()
    return {"value": nx * ny * steps / el, "unit": UNIT, "threads": orc.max_threads(),
            "sample": f"{nx}x{ny}" + ("" if crop is None else f" crop of {p.nx}x{p.ny}") + f", {steps} steps",
            "seconds": el}


def per_config(lbm, device, hbm, peak_ops):
    """Each configuration of the benchmark set on the GPU (and the oracle on the host):
    Sod 200x4 (a full 2000-step solve), thermal Couette 4x200 at Pr 0.5, 1, 2 (step time alone and
    as one batch), the shock-interface 4096x1024 (FP64 and FP32 with rooflines); the 8192^2 shear
    layer is the headline line itself."""
    import torch
    from paper_1305_4736_gb300 import workloads as wl
    from oracle import oracle as orc
    cores = os.cpu_count() or 1
    out = {}
    # Sod: one full solve per precision
    p = wl.sod(200, 4)
    sod = {}
    for name, prec in (("fp64", lbm.LBM_FP64), ("fp32", lbm.LBM_FP32_DEV)):
        r = config_gpu(lbm, p, prec, p.steps, 200, device, hbm)
        r["solve_ms"] = r["ms_per_step"] * p.steps
        r["solves_per_s"] = 1e3 / r["solve_ms"]
        sod[name] = r
    sod["oracle"] = {"all_cores": oracle_rate(p, 1000, cores), "one_thread": oracle_rate(p, 1000, 1)}
    sod["note"] = "latency-bound (800 cells): time per step and per 2000-step solve, not a roofline"
    out["sod_200x4"] = sod
    # Couette: each Pr alone and the three as one batch (FP64)
    cou = {}
    probs = [wl.couette(Pr, nx=4, ny=200) for Pr in (0.5, 1.0, 2.0)]
    for Pr, q in zip((0.5, 1.0, 2.0), probs):
        cou[f"fp64_Pr{Pr:g}"] = config_gpu(lbm, q, lbm.LBM_FP64, 2000, 200, device, hbm)
    solvers = [lbm.Solver.from_problem(q, device=device) for q in probs]
    for sv, q in zip(solvers, probs):
        sv.init(*q.fields())
    b = lbm.Batch(solvers)
    b.step(200)
    stream = torch.cuda.current_stream(device)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    ev0.record(stream)
    b.step(2000)
    ev1.record(stream)
    torch.cuda.synchronize(device)
    b.close()
    for sv in solvers:
        sv.close()
    cou["fp64_batch_of_3_us_per_step"] = 1e3 * ev0.elapsed_time(ev1) / 2000
    cou["oracle"] = {"all_cores": oracle_rate(probs[1], 1000, cores), "one_thread": oracle_rate(probs[1], 1000, 1)}
    cou["note"] = ("latency-bound (800 cells); a converged solve from rest takes 1e6-1e7 steps "
                   "(viscous time H^2/nu = 1000 at s5 = 1e3)")
    out["couette_4x200"] = cou
    # shock-interface at full size
    p = wl.shock_interface()
    si = {"fp64": config_gpu(lbm, p, lbm.LBM_FP64, 20, 3, device, hbm, peak_ops),
          "fp32": config_gpu(lbm, p, lbm.LBM_FP32_DEV, 200, 5, device, hbm)}
    si["oracle"] = {"all_cores": oracle_rate(p, 2, cores), "one_thread": oracle_rate(p, 10, 1, crop=(512, 128))}
    out["shock_interface_4096x1024"] = si
    # shear layer: the oracle only (the GPU numbers are the headline and fp64 lines)
    p = wl.shear_layer(N_GRID)
    out["shear_layer_8192x8192"] = {"oracle": {"all_cores": oracle_rate(p, 2, cores, crop=(2048, 2048)),
                                               "one_thread": oracle_rate(p, 10, 1, crop=(256, 256))}}
    orc.set_threads(cores)
    return out


def field_errors(a, b):
    """FP32 moments a against FP64 moments b: L1 and max relative errors of rho, u (as a vector), T."""
    import numpy as np

    def rel(x, y):
        return {"l1": float(np.abs(x - y).sum() / np.abs(y).sum()), "max": float(np.abs(x - y).max() / np.abs(y).max())}
    du = np.hypot(a[1] - b[1], a[2] - b[2])
    un = np.hypot(b[1], b[2])
    return {"rho": rel(a[0], b[0]), "T": rel(a[3], b[3]),
            "u": {"l1": float(du.sum() / un.sum()), "max": float(du.max() / un.max())}}


def precision_study(lbm, p, device, steps, every=None, delta_every=None, periodic=False):
    """FP32 deviation mode against FP64 on the same fields over `steps` steps: L1 and max relative
    errors of rho, u, T after the run (and at every `every` steps, the worst), the Delta moments at
    every `delta_every` steps, the FP32 totals against the FP64 ones, and (doubly periodic grids,
    where the flux form conserves them) the drift of the totals in each precision."""
    import numpy as np
    every = every or steps
    sol = {prec: lbm.Solver.from_problem(p, precision=prec, device=device)
           for prec in (lbm.LBM_FP64, lbm.LBM_FP32_DEV)}
    for sv in sol.values():
        sv.init(*p.fields())
    t0 = {prec: sv.totals() for prec, sv in sol.items()}
    bufs = {prec: _pinned_fields(p.ny, p.nx, 4) for prec in sol}
    dbufs = {prec: pinned_like(np.zeros((16, p.ny, p.nx))) for prec in sol} if delta_every else None
    worst = {"rho": {"l1": 0.0, "max": 0.0}, "u": {"l1": 0.0, "max": 0.0}, "T": {"l1": 0.0, "max": 0.0}}
    dworst = 0.0
    series = []
    done = 0
    tstart = time.perf_counter()
    while done < steps:
        n = min(every, steps - done)
        for sv in sol.values():
            sv.step(n)
        done += n
        want_delta = bool(delta_every) and done % delta_every == 0
        m = {}
        for prec, sv in sol.items():
            f = bufs[prec]
            d = dbufs[prec][0] if want_delta else None
            rc = lbm.lbm_moments(sv.h, f[0][0], f[1][0], f[2][0], f[3][0], d)
            if rc != 0:
                raise RuntimeError(f"lbm_moments failed ({rc}) at step {done}")
            m[prec] = [x[0] for x in f]
        e = field_errors(m[lbm.LBM_FP32_DEV], m[lbm.LBM_FP64])
        if done % 500 == 0 or done == steps:
            series.append({"step": done, **{k: {"l1": e[k]["l1"], "max": e[k]["max"]} for k in ("rho", "u", "T")}})
        for k in worst:
            for q in ("l1", "max"):
                worst[k][q] = max(worst[k][q], e[k][q])
        if want_delta:
            d32, d64 = dbufs[lbm.LBM_FP32_DEV][0][4:], dbufs[lbm.LBM_FP64][0][4:]
            dworst = max(dworst, float(np.abs(d32 - d64).sum() / max(np.abs(d64).sum(), 1e-300)))
    t1 = {prec: sv.totals() for prec, sv in sol.items()}
    for sv in sol.values():
        sv.close()
    a, b = t1[lbm.LBM_FP32_DEV], t1[lbm.LBM_FP64]
    out = {"steps": steps, "final": e, "worst_over_checkpoints": worst, "checkpoint_every": every,
           "series_every_500": series,
           "totals_fp32_vs_fp64": {"mass": abs(a[0] - b[0]) / abs(b[0]), "momentum_x": abs(a[1] - b[1]) / abs(b[0]),
                                   "momentum_y": abs(a[2] - b[2]) / abs(b[0]), "energy": abs(a[3] - b[3]) / abs(b[3])},
           "budget": {"l1": 1e-4, "max": 1e-3, "totals_drift": 1e-6},
           "seconds": time.perf_counter() - tstart}
    ok = (max(worst[k]["l1"] for k in worst) <= 1e-4 and max(worst[k]["max"] for k in worst) <= 1e-3
          and all(np.isfinite([out["final"][k][q] for k in ("rho", "u", "T") for q in ("l1", "max")])))
    if periodic:   # the flux form conserves the totals exactly on a doubly periodic grid
        out["totals_drift"] = {"fp32": totals_drift(t0[lbm.LBM_FP32_DEV], a, steps),
                               "fp64": totals_drift(t0[lbm.LBM_FP64], b, steps)}
        ok = ok and max(v for k, v in out["totals_drift"]["fp32"].items() if k != "steps") <= 1e-6
    if delta_every:
        out["delta_every"] = delta_every
        out["delta_rows_5_16_l1_worst"] = dworst
    out["within_budget"] = bool(ok)
    return out


def guarded(fn, *a, **kw):
    """Run one measurement section; a failure is reported in the line instead of ending the run."""
    try:
        return fn(*a, **kw)
    except Exception as e:   # noqa: BLE001 -- reported, not swallowed
        return {"error": f"{type(e).__name__}: {e}"}


def finish(line, p, args, rank, world):
    if rank == 0 and args.mode == "both":
        import torch
        from paper_1305_4736_gb300 import lbm, workloads as wl
        dev = torch.cuda.current_device()
        peaks, _ = measured_peaks()
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        if not args.no_configs:
            line["configs"] = guarded(per_config, lbm, dev, hbm, lbm.lbm_peak_fp64(dev) / 2.0)
        if not args.no_precision_study:
            line["precision"] = {
                f"shear_layer_{p.nx}x{p.ny}": guarded(precision_study, lbm, p, dev, 2000, periodic=True),
                "shock_interface_4096x1024": guarded(precision_study, lbm, wl.shock_interface(), dev, 5000,
                                                     every=100, delta_every=500),
            }
    if rank == 0 and not args.no_batch:
        import torch
        line["batch"] = guarded(batch_measure, torch.cuda.current_device())
    if rank == 0 and args.serving_requests > 0:
        import torch
        line["serving"] = guarded(serving_measure, args.serving_requests, args.serving_steps,
                                  args.serving_max_grid[0], args.serving_max_grid[1], torch.cuda.current_device())
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
