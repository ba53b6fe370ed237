"""The paper's Sec. IV.A and IV.B runs on the GPU at their stated parameters (float64).

- Discontinuity test (Sec. IV.A, workloads.discontinuity: gamma = 2, dx = 1e-3,
  dt = 1e-5, t = 0.06): with the MC limiter the shock sits where the exact solution
  puts it (x = 0.5 + 2 t, speed 2 from the Hugoniot states), the gas ahead is untouched
  and the density overshoot behind the shock stays below 2e-3; with psi = 1
  (Lax-Wendroff) the shocked region oscillates, the overshoot being more than 20 times
  the MC one (the paper's comparison of Fig. 3).  The GPU run matches the oracle at the
  full 6000 steps (1e-10).
- Lax shock tube (Sec. IV.B, workloads.lax: dx = 3e-3, dt = 1e-5, rates 2e3 / 1e3 /
  1e5): the paper's parameters put the model in its unstable regime (s5 fifty times
  below the rates of the higher moments; left state T = 7.9).  Round-off is amplified in
  the rarefaction: computations that agree to 1e-14 at 500 steps separate exponentially
  (1e-11 at 1000, 1e-3 at 2000 steps), and the oracle with the initial temperature
  perturbed by 1e-12 goes non-finite by step 9000, so whether a run reaches the paper's
  t = 0.45 depends on its rounding.  The GPU run is therefore compared with the exact
  Riemann solution at t = 0.05 (5000 steps; mean absolute errors of rho, u, p below 0.01,
  the oracle giving 0.0063, 0.0080, 0.0076) and with the oracle over the first 500 steps
  (1e-10).
"""
import numpy as np
import pytest

from _gpu_helpers import fp64_errors, run_both
from oracle import riemann as R
from paper_1305_4736_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1305_4736_gb300 import build, lbm as L
    build.build()
    L.load()
    return L


def _gpu_rho(lbm, p):
    s = lbm.Solver.from_problem(p)
    s.init(*p.fields())
    s.step(p.steps)
    out = [a[0] for a in s.moments()]
    s.close()
    return out


def test_discontinuity_mc_against_oracle_and_exact(orc, lbm):
    p = wl.discontinuity()
    s, O = run_both(orc, lbm, p, p.steps)
    errs = fp64_errors(s, O)
    for k, v in errs.items():
        assert v <= TOL, f"{k}: {v:.3e} ({errs})"
    rho = s.moments()[0][0]
    s.close()
    x = (np.arange(p.nx) + 0.5) * p.dx
    r2 = p.meta["left"][0]
    xs = 0.5 + 2.0 * p.steps * p.dt
    cross = x[np.argmax(rho < 0.5 * (r2 + 1.0))]
    assert abs(cross - xs) <= 2 * p.dx
    assert np.abs(rho[x > xs + 0.05] - 1.0).max() <= 1e-12
    behind = rho[(x > 0.1) & (x < xs - 0.02)]
    assert behind.max() - r2 <= 2e-3


def test_discontinuity_lax_wendroff_oscillates(lbm):
    mc = _gpu_rho(lbm, wl.discontinuity(limiter=0))[0]
    lw = _gpu_rho(lbm, wl.discontinuity(limiter=1))[0]
    p = wl.discontinuity()
    x = (np.arange(p.nx) + 0.5) * p.dx
    r2 = p.meta["left"][0]
    region = (x > 0.1) & (x < 0.5 + 2.0 * p.steps * p.dt - 0.02)
    over_mc = mc[region].max() - r2
    over_lw = lw[region].max() - r2
    assert over_lw > 20 * max(over_mc, 1e-6), (over_mc, over_lw)


def test_lax_tube_follows_exact_solution(lbm):
    p = wl.lax()
    p.steps = 5000                                   # t = 0.05, inside the stable window
    rho, u, _, T = _gpu_rho(lbm, p)
    L, Rt = p.meta["left"], p.meta["right"]
    sol = R.solve((L[0], L[1], L[0] * L[3]), (Rt[0], Rt[1], Rt[0] * Rt[3]), 1.4)
    x = (np.arange(p.nx) + 0.5) * p.dx
    t = p.steps * p.dt
    re, ue, pe = sol.sample((x - 0.5 * p.nx * p.dx) / t)
    assert np.abs(rho - re).mean() <= 0.01
    assert np.abs(u - ue).mean() <= 0.01
    assert np.abs(rho * T - pe).mean() <= 0.01
    # the end cells are outside the waves (uniform inflow states, drifting only by round-off)
    assert np.abs(rho[:5] - L[0]).max() <= 1e-8 and np.abs(rho[-5:] - Rt[0]).max() <= 1e-8


def test_lax_tube_against_oracle(orc, lbm):
    p = wl.lax()
    s, O = run_both(orc, lbm, p, 500)
    errs = fp64_errors(s, O)
    s.close()
    for k, v in errs.items():
        assert v <= TOL, f"{k}: {v:.3e} ({errs})"
