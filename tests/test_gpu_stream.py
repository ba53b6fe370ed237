"""GPU parity of the streaming step kernel (lbm_options.step_kernel = 5) and of the
persistent double-buffered TMA-staged kernel (step_kernel = 6, float32 only).

The kernel splits strips (256 columns) x rows evenly over its CTAs; a CTA's
range of rows may end inside one strip and continue at the top of the next, and
the last strip of a grid whose width is not a multiple of 256 is ragged.  The
grids below hit those cases: one strip with short ranges, several strips whose
ranges cross strip boundaries, ragged last strips, the minimum width of 128
columns, single-row and two-row grids.  Against the plain kernel the bar is
round-off of the storage precision (same arithmetic per value; the halo flow
velocities are summed in another order); against the oracle it is the float64
bar of 1e-10.
"""
import numpy as np
import pytest

from _gpu_helpers import fp64_errors
from paper_1305_4736_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-10
ROUNDOFF = {0: 1e-13, 1: 2e-5}


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1305_4736_gb300 import build, lbm as L
    build.build()
    L.load()
    return L


def _crop(p, nx, ny):
    p.nx, p.ny = nx, ny
    p.rho, p.ux, p.uy, p.T = (np.ascontiguousarray(a[:ny, :nx]) for a in (p.rho, p.ux, p.uy, p.T))
    return p


def _walls(p):
    p.bc = [(wl.BC_NEQ_WALL, 1.0, 0.0, 0.02, 1.01), (wl.BC_NEQ_WALL, 1.0, 0.0, -0.03, 0.99),
            (wl.BC_EQUILIBRIUM, 1.02, 0.01, 0.0, 1.0), (wl.BC_ZERO_GRADIENT, 0, 0, 0, 0)]
    return p


def _state_after(lbm, p, steps, precision, kernel, limiter=None):
    s = lbm.Solver(p.nx, p.ny, p.dx, p.dt, p.gamma, p.Pr, p.s, p.limiter if limiter is None else limiter,
                   p.bc, precision=precision, step_kernel=kernel)
    s.init(*p.fields())
    s.step(steps)
    out = s.get_state()
    s.close()
    return out


def _assert_roundoff(a, b, precision):
    assert np.isfinite(a).all()
    assert np.abs(a - b).max() <= ROUNDOFF[precision] * np.abs(b).max()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("limiter", [0, 1, 2])
def test_stream_matches_plain_one_strip(lbm, precision, limiter):
    p = wl.shock_interface(nx=150, ny=70, steps=60)          # one ragged strip, 3 CTAs of ~23 rows
    a = _state_after(lbm, p, 60, precision, 1, limiter)
    b = _state_after(lbm, p, 60, precision, 5, limiter)
    _assert_roundoff(b, a, precision)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nx,ny", [(600, 40), (300, 17), (513, 9), (128, 1), (129, 2), (1030, 33)])
def test_stream_matches_plain_spans_across_strips(lbm, precision, nx, ny):
    p = _crop(wl.shear_layer(max(nx, ny), seed=3, steps=40), nx, ny)
    a = _state_after(lbm, p, 40, precision, 1)
    b = _state_after(lbm, p, 40, precision, 5)
    _assert_roundoff(b, a, precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_stream_matches_plain_walls(lbm, precision):
    p = _walls(_crop(wl.shear_layer(300, ny=45), 290, 45))
    a = _state_after(lbm, p, 80, precision, 1)
    b = _state_after(lbm, p, 80, precision, 5)
    _assert_roundoff(b, a, precision)


@pytest.mark.parametrize("limiter", [0, 1, 2])
def test_stream_each_limiter_against_oracle(orc, lbm, limiter):
    p = wl.shock_interface(nx=280, ny=40, steps=120)
    s = lbm.Solver(p.nx, p.ny, p.dx, p.dt, p.gamma, p.Pr, p.s, limiter, p.bc, step_kernel=5)
    s.init(*p.fields())
    s.step(120)
    O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, limiter, p.bc)
    O.init(*p.fields())
    O.step(120)
    errs = fp64_errors(s, O)
    for k, v in errs.items():
        assert v <= TOL, f"{k}: {v:.3e} ({errs})"
    fo = O.get_state()
    assert np.abs(s.get_state() - fo).max() <= TOL * np.abs(fo).max()


def test_stream_walls_against_oracle(orc, lbm):
    p = _walls(_crop(wl.shear_layer(300, ny=30), 270, 30))
    s = lbm.Solver(p.nx, p.ny, p.dx, p.dt, p.gamma, p.Pr, p.s, p.limiter, p.bc, step_kernel=5)
    s.init(*p.fields())
    s.step(150)
    O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, p.limiter, p.bc)
    O.init(*p.fields())
    O.step(150)
    errs = fp64_errors(s, O)
    for k, v in errs.items():
        assert v <= TOL, f"{k}: {v:.3e} ({errs})"


def test_stream_rejects_narrow_grid(lbm):
    p = wl.shock_interface(nx=100, ny=20, steps=1)
    with pytest.raises(lbm.LbmError):
        lbm.Solver(p.nx, p.ny, p.dx, p.dt, p.gamma, p.Pr, p.s, p.limiter, p.bc, step_kernel=5)


def test_stream_no_copy_wait_ran_out(lbm):
    """A run of the streaming kernel leaves its copy-wait error flag clear (lbm_moments reads
    the flag back and reports LBM_ERR_TIMEOUT when a bounded wait ran out)."""
    p = wl.shear_layer(1024, seed=5, steps=50)
    s = lbm.Solver.from_problem(p, precision=1, step_kernel=5)
    s.init(*p.fields())
    s.step(50)
    rho, u, v, T = s.moments()
    s.close()
    assert np.isfinite(rho).all() and np.isfinite(T).all()


# ------------------------------------------------ persistent double-buffered TMA-staged kernel
@pytest.mark.parametrize("limiter", [0, 1, 2])
@pytest.mark.parametrize("nx,ny", [(150, 70), (32, 16), (61, 45), (600, 40), (1030, 33)])
def test_pipe_matches_plain(lbm, limiter, nx, ny):
    p = _crop(wl.shear_layer(max(nx, ny), seed=4, steps=40), nx, ny)
    a = _state_after(lbm, p, 40, 1, 1, limiter)
    b = _state_after(lbm, p, 40, 1, 6, limiter)
    _assert_roundoff(b, a, 1)


def test_pipe_matches_plain_walls(lbm):
    p = _walls(_crop(wl.shear_layer(300, ny=45), 290, 45))
    a = _state_after(lbm, p, 80, 1, 1)
    b = _state_after(lbm, p, 80, 1, 6)
    _assert_roundoff(b, a, 1)


def test_pipe_is_float32_only(lbm):
    p = wl.shock_interface(nx=150, ny=70, steps=1)
    with pytest.raises(lbm.LbmError):
        lbm.Solver(p.nx, p.ny, p.dx, p.dt, p.gamma, p.Pr, p.s, p.limiter, p.bc, precision=0, step_kernel=6)


# ------------------------------------------------ TMA-staged kernel across state changes
def test_tma_kernel_across_set_state_and_batch_steps(lbm):
    """The float32 TMA-staged kernel on a ragged doubly periodic grid, stepped in uneven chunks
    with a get_state / set_state round trip and a batch step in between, matches the plain
    kernel to round-off."""
    p = _crop(wl.shear_layer(160, seed=8, steps=60), 150, 70)     # ragged against 32 x 16 tiles
    ref = lbm.Solver.from_problem(p, precision=1, step_kernel=1)
    ref.init(*p.fields())
    s = lbm.Solver.from_problem(p, precision=1, step_kernel=2)
    s.init(*p.fields())
    for chunk in (7, 13, 1):
        ref.step(chunk)
        s.step(chunk)
    mid = s.get_state()
    s.set_state(mid)
    ref.set_state(ref.get_state())
    b = lbm.Batch([s])
    b.step(3)
    b.close()
    ref.step(3)
    s.step(36)
    ref.step(36)
    got, want = s.get_state(), ref.get_state()
    s.close()
    ref.close()
    assert np.isfinite(got).all()
    assert np.abs(got - want).max() <= ROUNDOFF[1] * np.abs(want).max()


def test_bounded_wait_runs_out_without_a_fault(lbm):
    """A wait on an mbarrier phase that nothing completes (the kernels' own bounded wait) gives
    up at its 2 s limit: the kernel records it, the host reads LBM_ERR_TIMEOUT, and the device
    stays usable for the next solve."""
    rc, ms = lbm.lbm_wait_selftest(0)
    assert rc == lbm.LBM_ERR_TIMEOUT
    assert 1800.0 <= ms <= 10000.0
    p = wl.shear_layer(256, seed=2, steps=5)
    s = lbm.Solver.from_problem(p, precision=1)
    s.init(*p.fields())
    s.step(5)
    rho = s.moments()[0]
    s.close()
    assert np.isfinite(rho).all()
