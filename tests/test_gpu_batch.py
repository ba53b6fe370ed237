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
    assert choice in (1, 2, 3, 4, 5, 6, 7, 8, 9)
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
    """A float64 1280 x 1024 member on the streaming kernel runs that kernel inside the batch's
    graph, and a float32 640 x 512 member on the tile kernel goes to the batched tile kernel:
    both bit-identical to stepping them alone.  The float64 Sod member, on the plain kernel,
    shares the packed plain kernel.
    Stepping a member alone an odd number of times between batch steps flips its buffer
    parity, and the batch recaptures its graph."""
    specs = [(wl.shear_layer(640, ny=512, seed=3), 1, 0), (wl.shear_layer(1280, ny=1024, seed=4), 0, 5),
             (wl.sod(200, 4), 0, 7), (wl.shear_layer(96, ny=40, seed=5), 1, 0)]

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


def _tma_mix():
    """Uneven grids for the batched TMA-staged kernels: float32 and float64 (double-float),
    from one tile to many, ragged edges, walls with the energy-flux correction, every limiter."""
    out = []
    for k, (nx, ny) in enumerate([(32, 32), (48, 40), (100, 70), (333, 129), (640, 256)]):
        out.append((wl.shear_layer(nx, ny=ny, seed=11 + k), 1, (0, 1, 2)[k % 3]))
        out.append((wl.shock_interface(nx=nx, ny=ny, steps=1), 0, (2, 0, 1)[k % 3]))
    q = wl.shear_layer(96, ny=66, seed=21)
    q.bc = [(wl.BC_NEQ_WALL, 1.0, 0.0, 0.02, 1.01), (wl.BC_NEQ_WALL, 1.0, 0.0, -0.03, 0.99),
            (wl.BC_EQUILIBRIUM, 1.02, 0.01, 0.0, 1.0), (wl.BC_ZERO_GRADIENT, 0, 0, 0, 0)]
    out.append((q, 0, 0))
    out.append((q, 1, 0))
    # float64 grids of 4 to 31 rows: the double-float kernel on narrow 32 x 4 tiles
    for k, (nx, ny) in enumerate([(32, 4), (100, 13), (250, 31)]):
        out.append((wl.shock_interface(nx=nx, ny=ny, steps=1), 0, (0, 1, 2)[k]))
    return out


def _tma_kernel(s):
    """The kernel a member of the TMA-staged mix runs alone: float32 tiles; float64 32 x 32 tiles
    on grids of at least two thirds of a wave of them, else narrow 32 x 4 tiles (in the batch,
    every float64 member whose grid takes 32 x 32 tiles steps on those)."""
    import torch
    if s.precision == 1:
        return 2
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tiles = ((s.nx + 31) // 32) * ((s.ny + 31) // 32)
    return 8 if s.ny >= 32 and 3 * tiles >= 2 * sms else 9


def test_batched_tma_kernels_equal_solo_bit_for_bit(lbm):
    """Members on the tile kernel (float32) and the double-float kernel (float64) step in the
    batched TMA-staged launches with the arithmetic of their single-grid kernels: bit-identical
    to stepping alone, over a graph replay, an odd step and a solo step in between."""
    probs = _tma_mix()
    batched = [_solver(lbm, p, prec, lim, 0) for p, prec, lim in probs]
    solo = [_solver(lbm, p, prec, lim, 0) for p, prec, lim in probs]
    for s in batched:
        assert s.step_kernel == _tma_kernel(s)
    b = lbm.Batch(batched)
    b.step(9)
    batched[3].step(1)
    solo[3].step(1)
    b.step(2)
    for s in solo:
        s.step(11)
    for (p, prec, lim), x, y in zip(probs, batched, solo):
        assert np.array_equal(x.get_state(), y.get_state()), (p.name, p.nx, p.ny, prec, lim)
    b.close()


def test_batched_tma_members_against_oracle(orc, lbm):
    """Each member of a mixed batch after 60 batched steps against the oracle: float64
    (double-float kernel) to 1e-10 on rho, u, T; float32 (tile kernel) within L1 1e-4 and
    max 1e-3."""
    from _gpu_helpers import l1_rel, max_rel
    probs = _tma_mix()
    batched = [_solver(lbm, p, prec, lim, 0) for p, prec, lim in probs]
    b = lbm.Batch(batched)
    b.step(60)
    b.close()
    for (p, prec, lim), s in zip(probs, batched):
        O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, lim, p.bc)
        O.init(*p.fields())
        O.step(60)
        if prec == 0:
            errs = fp64_errors(s, O)
            assert max(errs.values()) <= 1e-10, (p.name, p.nx, p.ny, lim, errs)
        else:
            g, r = s.moments(), O.moments()
            for a, c in ((g[0], r[0]), (g[3], r[3])):
                assert l1_rel(a, c) <= 1e-4 and max_rel(a, c) <= 1e-3, (p.name, p.nx, p.ny, lim)
            du = np.hypot(g[1] - r[1], g[2] - r[2])
            un = np.hypot(r[1], r[2])
            assert du.sum() / un.sum() <= 1e-4 and du.max() / un.max() <= 1e-3, (p.name, p.nx, p.ny, lim)
        s.close()


def test_batched_tma_launches_split_past_the_parameter_block(lbm):
    """A batch group with more tile-kernel members than one launch's parameter block holds
    (128 grids) steps them in several launches: 140 float32 grids and 133 float64 grids of
    one to six tiles each, with different sizes, limiters and seeds, bit-identical to stepping
    each alone, over a graph replay, an odd step and a member stepped alone in between."""
    probs = []
    rng = np.random.default_rng(5)
    for k in range(140):
        nx, ny = int(rng.choice([32, 40, 64, 96])), int(rng.choice([16, 20, 32, 48]))
        probs.append((wl.shear_layer(nx, ny=ny, seed=100 + k), 1, 0))
    for k in range(133):
        nx, ny = int(rng.choice([32, 48, 64])), int(rng.choice([32, 40, 64]))
        probs.append((wl.shear_layer(nx, ny=ny, seed=300 + k), 0, 0))
    batched = [_solver(lbm, p, prec, lim, 0) for p, prec, lim in probs]
    solo = [_solver(lbm, p, prec, lim, 0) for p, prec, lim in probs]
    for s in batched:
        assert s.step_kernel == _tma_kernel(s)
    b = lbm.Batch(batched)
    b.step(4)
    batched[130].step(1)
    solo[130].step(1)
    batched[270].step(1)
    solo[270].step(1)
    b.step(3)
    for s in solo:
        s.step(7)
    for k, (x, y) in enumerate(zip(batched, solo)):
        assert np.array_equal(x.get_state(), y.get_state()), (k, probs[k][0].nx, probs[k][0].ny)
    b.close()
    for s in batched + solo:
        s.close()
