"""Scheduling logic of the serving loop, on the host with a fake backend and a fake clock:
every request finishes with its own step count, admission follows arrival order and never
exceeds the memory budget, later arrivals join while earlier solves are still resident
(continuous batching), and the batch is rebuilt when its membership changes."""
import numpy as np
import pytest

from paper_1305_4736_gb300 import serving, workloads as wl


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeSolver:
    def __init__(self, p, prec):
        self.p, self.prec, self.steps = p, prec, 0


class FakeBackend:
    def __init__(self, clock, step_cost=1e-6):
        self.clock, self.cost = clock, step_cost
        self.batches = []
        self.resident = 0

    def footprint(self, p, precision):
        return p.cells * (4 if precision else 8) * 32

    def create(self, p, precision):
        self.resident += 1
        return FakeSolver(p, precision)

    def batch(self, solvers):
        self.batches.append([id(s) for s in solvers])
        return list(solvers)

    def step(self, batch, n):
        self.clock.t += self.cost * n * sum(s.p.cells for s in batch)
        for s in batch:
            s.steps += n

    def step_one(self, s, n):
        s.steps += n

    def finish(self, s):
        self.resident -= 1
        return (s.steps,)

    def close_batch(self, b):
        pass


def _requests(n=24, seed=3):
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    for i in range(n):
        t += rng.exponential(0.002)
        p = wl.sod(int(rng.integers(20, 200)) * 2, 4)
        p.steps = int(rng.integers(50, 400))
        reqs.append({"id": i, "kind": "riemann", "arrival": t, "problem": p, "precision": int(i % 2)})
    return reqs


@pytest.mark.parametrize("realtime", [True, False])
def test_every_request_finishes_with_its_steps(realtime):
    clk = FakeClock()
    be = FakeBackend(clk)
    reqs = _requests()
    res, st = serving.Engine(be, budget_bytes=10 ** 9, chunk=64, realtime=realtime).run(reqs, clk, clk.sleep)
    assert [r.id for r in res] == list(range(len(reqs)))
    for r, q in zip(res, reqs):
        assert r.moments == (q["problem"].steps,)
        assert r.done >= r.admitted >= 0 and r.latency >= 0
        if realtime:
            assert r.admitted >= q["arrival"]
    assert be.resident == 0 and st.solves == len(reqs)
    assert st.cell_updates == sum(q["problem"].steps * q["problem"].cells for q in reqs)


def test_budget_respected_and_arrival_order():
    clk = FakeClock()
    be = FakeBackend(clk)
    reqs = _requests(30, seed=5)
    budget = 3 * max(be.footprint(q["problem"], q["precision"]) for q in reqs)
    res, st = serving.Engine(be, budget_bytes=budget, chunk=32).run(reqs, clk, clk.sleep)
    assert st.max_resident_bytes <= budget
    adm = sorted(res, key=lambda r: r.admitted)
    assert [r.id for r in adm] == sorted(r.id for r in res)      # no request overtakes an earlier one


def test_continuous_batching_overlaps_requests():
    clk = FakeClock()
    be = FakeBackend(clk, step_cost=1e-5)
    reqs = _requests(16, seed=7)
    res, st = serving.Engine(be, budget_bytes=10 ** 9, chunk=16).run(reqs, clk, clk.sleep)
    assert st.max_resident_solves >= 3
    # some request was admitted while another, admitted earlier, was still running
    overlap = any(a.admitted < b.admitted < a.done for a in res for b in res if a is not b)
    assert overlap
    sizes = [len(b) for b in be.batches]
    assert len(set(sizes)) > 1                      # membership changed and the batch was rebuilt


def test_request_larger_than_budget_is_rejected():
    clk = FakeClock()
    be = FakeBackend(clk)
    reqs = _requests(2)
    with pytest.raises(ValueError):
        serving.Engine(be, budget_bytes=10).run(reqs, clk, clk.sleep)
