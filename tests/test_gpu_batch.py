"""Batched stepping (lbm_batch) and the kernel autotuner on the GPU.

- A batch of uneven grids mixing precisions, limiters and boundary kinds gives, for every
  problem, the state of that problem stepped alone (same per-cell arithmetic; multiply-add
  contraction may differ, so round-off of the storage precision), over odd step counts
  (graph replay of step pairs plus a single step) and with solo steps interleaved.
- A grid's result does not depend on the other members of its batch (bit for bit).
- lbm_autotune does not advance the state, and the kernel it keeps still matches the oracle.
"""
import numpy as np
import pytest

from _gpu_helpers import fp64_errors
from paper_1305_4736_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1305_4736_gb300 import build, lbm as L
    build.build()
    L.load()
    return L


def _problems():
    out = []
    out.append((wl.sod(200, 4), 0, None))
    out.append((wl.couette(0.5, nx=4, ny=200), 0, None))
    out.append((wl.shock_interface(nx=70, ny=20, steps=1), 1, None))
    out.append((wl.shear_layer(100, ny=70), 0, 1))              # Lax-Wendroff
    out.append((wl.shock_interface(nx=45, ny=37, steps=1), 0, 2))   # upwind
    p = wl.shear_layer(64, ny=1)
    p.nx, p.ny = 1, 1
    p.rho, p.ux, p.uy, p.T = (np.ascontiguousarray(a[:1, :1]) for a in (p.rho, p.ux, p.uy, p.T))
    out.append((p, 1, None))
    q = wl.shear_layer(64, ny=33)
    q.nx = 40
    q.rho, q.ux, q.uy, q.T = (np.ascontiguousarray(a[:, :40]) for a in (q.rho, q.ux, q.uy, q.T))
    q.bc = [(wl.BC_NEQ_WALL, 1.0, 0.0, 0.02, 1.01), (wl.BC_NEQ_WALL, 1.0, 0.0, -0.03, 0.99),
            (wl.BC_EQUILIBRIUM, 1.02, 0.01, 0.0, 1.0), (wl.BC_ZERO_GRADIENT, 0, 0, 0, 0)]
    out.append((q, 1, None))
    return out


def _solver(lbm, p, prec, lim, kernel):
    s = lbm.Solver(p.nx, p.ny, p.dx, p.dt, p.gamma, p.Pr, p.s, p.limiter if lim is None else lim, p.bc,
                   precision=prec, step_kernel=kernel)
    s.init(*p.fields())
    return s


ROUNDOFF = {0: 1e-13, 1: 2e-5}


def test_batch_equals_solo_to_roundoff(lbm):
    probs = _problems()
    batched = [_solver(lbm, p, prec, lim, 1) for p, prec, lim in probs]
    solo = [_solver(lbm, p, prec, lim, 1) for p, prec, lim in probs]
    b = lbm.Batch(batched)
    b.step(37)                       # 18 graph replays of two steps + one single step
    batched[2].step(3)               # a solo step between batch steps
    solo[2].step(3)
    b.step(1)
    b.step(20)
    for s in solo:
        s.step(58)
    for (p, prec, lim), x, y in zip(probs, batched, solo):
        assert x.step_count == y.step_count
        a, c = x.get_state(), y.get_state()
        assert np.abs(a - c).max() <= ROUNDOFF[prec] * np.abs(c).max(), (p.name, prec, lim)
    b.close()


def test_batch_member_result_independent_of_mix(lbm):
    probs = _problems()
    mix = [_solver(lbm, p, prec, lim, 1) for p, prec, lim in probs]
    b = lbm.Batch(mix)
    b.step(25)
    for k, (p, prec, lim) in enumerate(probs):
        alone = _solver(lbm, p, prec, lim, 1)
        one = lbm.Batch([alone])
        one.step(25)
        assert np.array_equal(alone.get_state(), mix[k].get_state()), (p.name, prec, lim)
        one.close()
    b.close()


def test_batch_rejects_bad_sets(lbm):
    p = wl.sod(200, 2)
    s = _solver(lbm, p, 0, None, 1)
    with pytest.raises(lbm.LbmError):
        lbm.Batch([s, s])
    t = lbm.Solver.from_problem(p)             # never initialised
    b = lbm.Batch([s, t])
    with pytest.raises(lbm.LbmError):
        b.step(2)
    b.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_autotune_keeps_state_and_parity(orc, lbm, prec):
    p = wl.shear_layer(128, ny=96)
    s = lbm.Solver.from_problem(p, precision=prec)
    s.init(*p.fields())
    s.step(10)
    before = s.get_state()
    choice = s.autotune(3)
    assert choice in (1, 2, 3, 4, 5, 6, 7)
    assert s.step_kernel == choice
    assert np.array_equal(s.get_state(), before)
    assert s.step_count == 10
    s.step(90)
    if prec == 0:
        O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, p.limiter, p.bc)
        O.init(*p.fields())
        O.step(100)
        errs = fp64_errors(s, O)
        assert max(errs.values()) <= 1e-10, errs


def test_batch_runs_large_members_on_their_own_kernels(lbm):
    """Members whose own kernel is TMA-staged and fills a wave of its tiles (here a float32
    640 x 512 grid and a float64 1280 x 1024 grid) run that kernel inside the batch's graph:
    bit-identical to stepping them alone. The small members share the packed tile kernel.
    Stepping a large member alone an odd number of times between batch steps flips its
    buffer parity, and the batch recaptures its graph."""
    specs = [(wl.shear_layer(640, ny=512, seed=3), 1, 0), (wl.shear_layer(1280, ny=1024, seed=4), 0, 5),
             (wl.sod(200, 4), 0, 0), (wl.shear_layer(96, ny=40, seed=5), 1, 0)]

    def make():
        out = []
        for p, prec, kernel in specs:
            s = lbm.Solver.from_problem(p, precision=prec, step_kernel=kernel)
            s.init(*p.fields())
            out.append(s)
        return out

    batched, solo = make(), make()
    assert batched[0].step_kernel == 2 and batched[1].step_kernel == 5
    b = lbm.Batch(batched)
    b.step(6)
    batched[0].step(1)
    b.step(4)
    b.step(3)
    solo[0].step(1)
    for s in solo:
        s.step(13)
    for k, ((p, prec, _), x, y) in enumerate(zip(specs, batched, solo)):
        assert x.step_count == y.step_count
        got, want = x.get_state(), y.get_state()
        if k < 2:
            assert np.array_equal(got, want), p.name
        else:
            assert np.abs(got - want).max() <= ROUNDOFF[prec] * np.abs(want).max(), p.name
    b.close()
    for s in batched + solo:
        s.close()
