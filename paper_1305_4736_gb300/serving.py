"""Continuous-batching serving loop for FDLBM solves.

Requests (Riemann, Couette, shock-interface problems of different sizes, gamma, Pr and
precision) arrive over time.  The engine:
  - admits a waiting request as soon as its device footprint (lbm_footprint: both
    population buffers) fits the memory budget next to the solves already resident;
  - keeps every admitted solve's state resident on the GPU and advances all of them
    together, a chunk of steps at a time, through one lbm_batch (one batched ghost-fill
    and one batched fused-step launch per precision/limiter group per step, replayed from
    a CUDA graph); the batch is rebuilt whenever its membership changes;
  - retires a solve when its steps are done: its moments (rho, u, v, T) are read back,
    its memory is released, and its time to result (completion - arrival) is recorded.
Requests that arrive while others run are admitted at the next chunk boundary, so their
work overlaps on the device with the solves already in flight.

The backend is injectable: `GpuBackend` drives liblbm.so; tests of the scheduling logic
use a host-only fake.
"""
from __future__ import annotations

import heapq
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Result:
    id: int
    kind: str
    precision: int
    cells: int
    steps: int
    arrival: float
    admitted: float
    done: float
    moments: tuple = ()

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class Stats:
    solves: int
    wall: float
    solves_per_s: float
    p50: float
    p99: float
    max_resident_bytes: int
    max_resident_solves: int
    cell_updates: int
    chunks: int
    extra: dict = field(default_factory=dict)


class GpuBackend:
    """liblbm.so through the ctypes binding (device memory from torch's caching allocator)."""

    def __init__(self, device: int = 0):
        from . import lbm
        self.lbm = lbm
        lbm.load()
        self.device = device

    def footprint(self, p, precision) -> int:
        return self.lbm.lbm_footprint(p.nx, p.ny, precision)

    def create(self, p, precision):
        s = self.lbm.Solver.from_problem(p, precision=precision, device=self.device)
        s.init(*p.fields())
        return s

    def batch(self, solvers):
        return self.lbm.Batch(solvers)

    def step(self, batch, n: int):
        batch.step(n)

    def step_one(self, solver, n: int):
        solver.step(n)

    def finish(self, solver):
        out = solver.moments()
        solver.close()
        return out

    def close_batch(self, batch):
        batch.close()


class Engine:
    def __init__(self, backend, budget_bytes: int = 64 << 30, chunk: int = 100, realtime: bool = True):
        self.backend = backend
        self.budget = int(budget_bytes)
        self.chunk = int(chunk)
        self.realtime = realtime

    def run(self, requests, clock=time.perf_counter, sleep=time.sleep):
        """requests: iterable of dicts {id, kind, arrival, problem, precision} (arrival in s from
        the start; with realtime=False every request is available at the start).
        Returns (results sorted by id, Stats)."""
        reqs = sorted(requests, key=lambda r: r["arrival"])
        for r in reqs:
            if self.backend.footprint(r["problem"], r["precision"]) > self.budget:
                raise ValueError(f"request {r['id']} needs more than the whole memory budget")
        t0 = clock()
        now = lambda: clock() - t0  # noqa: E731
        waiting = []           # (arrival, id, request) that have arrived
        pending = list(reqs)   # not yet arrived, sorted by arrival
        active = {}            # id -> dict(solver, left, req, admitted, bytes)
        results = []
        used = 0
        max_used = max_n = chunks = 0
        cell_updates = 0
        batch = None
        dirty = True
        while pending or waiting or active:
            t = now()
            while pending and (not self.realtime or pending[0]["arrival"] <= t):
                r = pending.pop(0)
                heapq.heappush(waiting, (r["arrival"], r["id"], r))
            # admit in arrival order while the footprint fits (no overtaking)
            while waiting:
                r = waiting[0][2]
                need = self.backend.footprint(r["problem"], r["precision"])
                if used + need > self.budget:
                    break
                heapq.heappop(waiting)
                s = self.backend.create(r["problem"], r["precision"])
                active[r["id"]] = {"solver": s, "left": int(r["problem"].steps), "req": r,
                                   "admitted": now(), "bytes": need}
                used += need
                dirty = True
            max_used = max(max_used, used)
            max_n = max(max_n, len(active))
            if not active:
                if pending and self.realtime:
                    wait = pending[0]["arrival"] - now()
                    if wait > 0:
                        sleep(min(wait, 0.05))
                continue
            if dirty:
                if batch is not None:
                    self.backend.close_batch(batch)
                batch = self.backend.batch([a["solver"] for a in active.values()])
                dirty = False
            n = min(self.chunk, min(a["left"] for a in active.values()))
            self.backend.step(batch, n)
            chunks += 1
            for a in active.values():
                a["left"] -= n
                cell_updates += n * a["req"]["problem"].cells
            done_ids = [i for i, a in active.items() if a["left"] == 0]
            if done_ids:
                self.backend.close_batch(batch)
                batch = None
                dirty = True
                for i in done_ids:
                    a = active.pop(i)
                    m = self.backend.finish(a["solver"])
                    r = a["req"]
                    results.append(Result(r["id"], r["kind"], r["precision"], r["problem"].cells,
                                          int(r["problem"].steps), r["arrival"], a["admitted"], now(), m))
                    used -= a["bytes"]
        if batch is not None:
            self.backend.close_batch(batch)
        wall = now()
        lat = np.array([r.latency for r in results]) if results else np.zeros(1)
        stats = Stats(len(results), wall, len(results) / wall if wall > 0 else 0.0,
                      float(np.percentile(lat, 50)), float(np.percentile(lat, 99)), max_used, max_n,
                      cell_updates, chunks)
        return sorted(results, key=lambda r: r.id), stats


def one_at_a_time(backend, requests, precision=None, clock=time.perf_counter):
    """Solve the requests one after the other with plain per-context stepping (no batching).
    precision=None keeps each request's precision; 0 forces float64.  Returns (wall s, results)."""
    t0 = clock()
    out = []
    for r in sorted(requests, key=lambda r: r["id"]):
        prec = r["precision"] if precision is None else precision
        s = backend.create(r["problem"], prec)
        backend.step_one(s, int(r["problem"].steps))
        out.append(backend.finish(s))
    return clock() - t0, out
