"""GPU parity on grids with dy != dx (lbm_options.dy).

The y projection of the convection uses the Courant numbers |v_iy| dt / dy and the
y differences of the energy-flux correction divide by 2 dy (Sec. III, Sec. II).  The
oracle's handling of dy is pinned on the CPU (tests/test_oracle_aniso.py); here every
fused-step kernel is compared with it (float64 bar 1e-10) or with the plain kernel
(round-off of the storage precision), with the gradient correction active (Pr != 1),
for dy below and above dx, every limiter, walls, and a batch that mixes spacings.
"""
import numpy as np
import pytest

from _gpu_helpers import fp64_errors, l1_rel, max_rel, run_both, vel_max_rel
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


def _aniso(nx, ny, ratio, seed=9, walls=False):
    """Shear layer on an nx x ny grid with dy = ratio * dx (dx = 1/nx, dt = 1e-5, Pr = 0.71)."""
    p = wl.shear_layer(max(nx, ny), seed=seed)
    p.nx, p.ny = nx, ny
    p.rho, p.ux, p.uy, p.T = (np.ascontiguousarray(a[:ny, :nx]) for a in (p.rho, p.ux, p.uy, p.T))
    p.dx = 1.0 / nx
    p.dy = ratio * p.dx
    if walls:
        p.bc = [(wl.BC_NEQ_WALL, 1.0, 0.0, 0.02, 1.01), (wl.BC_NEQ_WALL, 1.0, 0.0, -0.03, 0.99),
                (wl.BC_EQUILIBRIUM, 1.02, 0.01, 0.0, 1.0), (wl.BC_ZERO_GRADIENT, 0, 0, 0, 0)]
    return p


def _solver(lbm, p, precision, kernel, limiter=None):
    return lbm.Solver(p.nx, p.ny, p.dx, p.dt, p.gamma, p.Pr, p.s, p.limiter if limiter is None else limiter,
                      p.bc, precision=precision, step_kernel=kernel, dy=p.dy)


def _state_after(lbm, p, steps, precision, kernel, limiter=None):
    s = _solver(lbm, p, precision, kernel, limiter)
    s.init(*p.fields())
    s.step(steps)
    out = s.get_state()
    s.close()
    return out


@pytest.mark.parametrize("ratio", [0.6, 1.7])
@pytest.mark.parametrize("kernel", [0, 1, 2, 5])
def test_fp64_against_oracle(orc, lbm, ratio, kernel):
    p = _aniso(160, 40, ratio)
    s = _solver(lbm, p, 0, kernel)
    s.init(*p.fields())
    s.step(150)
    O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, p.limiter, p.bc, dy=p.dy)
    O.init(*p.fields())
    O.step(150)
    errs = fp64_errors(s, O)
    for k, v in errs.items():
        assert v <= TOL, f"{k}: {v:.3e} ({errs})"
    fo = O.get_state()
    assert np.abs(s.get_state() - fo).max() <= TOL * np.abs(fo).max()


@pytest.mark.parametrize("limiter", [1, 2])
def test_fp64_limiters_and_walls_against_oracle(orc, lbm, limiter):
    p = _aniso(150, 36, 0.75, walls=True)
    s, O = run_both(orc, lbm, p, 120, limiter=limiter)
    errs = fp64_errors(s, O)
    for k, v in errs.items():
        assert v <= TOL, f"{k}: {v:.3e} ({errs})"


@pytest.mark.parametrize("kernel", [2, 5, 6])
def test_fp32_kernels_match_plain(lbm, kernel):
    p = _aniso(300, 45, 1.3, walls=True)
    a = _state_after(lbm, p, 60, 1, 1)
    b = _state_after(lbm, p, 60, 1, kernel)
    assert np.isfinite(b).all()
    assert np.abs(b - a).max() <= ROUNDOFF[1] * np.abs(a).max()


def test_fp32_deviation_budget_against_oracle(orc, lbm):
    p = _aniso(128, 64, 0.8)
    s, O = run_both(orc, lbm, p, 300, precision=lbm.LBM_FP32_DEV)
    g, r = s.moments(), O.moments()
    for a, b in ((g[0], r[0]), (g[3], r[3])):
        assert l1_rel(a, b) <= 1e-4 and max_rel(a, b) <= 1e-3
    assert vel_max_rel(g[1], g[2], r[1], r[2]) <= 1e-3


def test_totals_scale_with_dx_dy(orc, lbm):
    p = _aniso(96, 32, 1.5)
    s, O = run_both(orc, lbm, p, 20)
    t, to = np.asarray(s.totals()), np.asarray(O.totals())
    assert np.abs(t - to).max() <= 1e-12 * np.abs(to).max()


def test_batch_mixes_spacings(lbm):
    probs = [_aniso(100, 30, 0.7, seed=1), _aniso(64, 48, 1.9, seed=2), _aniso(80, 20, 1.0, seed=3)]
    solo = [_state_after(lbm, p, 33, 0, 1) for p in probs]
    sols = []
    for p in probs:
        s = _solver(lbm, p, 0, 1)
        s.init(*p.fields())
        sols.append(s)
    b = lbm.Batch(sols)
    b.step(33)
    b.close()
    for s, want in zip(sols, solo):
        got = s.get_state()
        s.close()
        assert np.abs(got - want).max() <= ROUNDOFF[0] * np.abs(want).max()
