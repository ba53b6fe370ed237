"""The non-equilibrium study of Sec. V on the GPU: a Mach-sqrt2 shock (gamma = 2) crosses
a heavy -> light interface; at t = 0.3 the centre line shows a reflected rarefaction, the
material interface and the transmitted shock.  The paper states (discussion of Fig. 6):
  - Delta*_6 is negative at the rarefaction and positive at the shock;
  - the peak deviations at the shock are larger than at the other two waves;
  - Delta*_10 is of the same order at the material interface and the shock and much larger
    than at the rarefaction;
  - Delta*_5, Delta*_7, Delta*_11 have small amplitudes;
  - away from the waves the system is back in equilibrium.
Wave positions come from the exact Riemann solution of the shock-interface interaction.
The GPU's Delta* also matches the oracle's (FP64 parity) after the first 2000 steps.
"""
import numpy as np
import pytest

from oracle import riemann
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


def _wave_positions(p, t):
    """Reflected rarefaction (head, tail), contact and transmitted shock at time t."""
    rs, us, ps = p.meta["shocked"]
    t_hit = (p.meta["x_interface"] - p.meta["x_shock"]) / p.meta["shock_speed"]
    sol = riemann.solve((rs, us, ps), p.meta["light"], p.gamma)
    lh, lt, c, rt, rh = sol.wave_speeds()
    dt = t - t_hit
    x0 = p.meta["x_interface"]
    return x0 + lh * dt, x0 + lt * dt, x0 + c * dt, x0 + rh * dt


def test_sec5_delta_star_signs_and_ordering(lbm):
    p = wl.shock_heavy_light()
    s = lbm.Solver.from_problem(p)
    s.init(*p.fields())
    s.step(p.steps)
    ds = s.moments_central()[:, p.ny // 2, :]          # centre line y = 0.005
    rho = s.moments()[0][p.ny // 2]
    s.close()
    assert np.all(np.isfinite(ds)) and np.all(rho > 0)
    x = (np.arange(p.nx) + 0.5) * p.dx
    xr_head, xr_tail, xc, xs = _wave_positions(p, p.steps * p.dt)
    assert 0.0 < xr_head < xr_tail < xc < xs < 1.2
    w = 0.02
    rare = (x > xr_head - w) & (x < xr_tail + w)
    cont = np.abs(x - xc) < w
    shock = np.abs(x - xs) < w
    quiet = np.ones_like(x, bool)
    for a, b in ((xr_head - 2 * w, xr_tail + 2 * w), (xc - 2 * w, xc + 2 * w), (xs - 2 * w, xs + 2 * w)):
        quiet &= ~((x > a) & (x < b))
    quiet &= (x > 0.05) & (x < 1.15)
    d6, d10 = ds[5], ds[9]
    peak = np.abs(d6).max()
    noise6 = np.abs(d6[quiet]).max()
    assert d6[rare].min() < -5.0 * noise6                # negative at the rarefaction (13x the background)
    assert d6[rare].max() < 0.1 * -d6[rare].min()        # ... and not positive there
    assert d6[shock].max() > 0.5 * peak                  # positive (and largest) at the shock
    assert d6[shock].max() > 10.0 * -d6[rare].min()      # the shock's peak dominates
    assert d6[shock].max() > 10.0 * np.abs(d6[cont]).max()
    a10_s, a10_c, a10_r = (np.abs(d10[m]).max() for m in (shock, cont, rare))
    assert a10_s > a10_r and a10_c > a10_r               # much larger than at the rarefaction
    assert 0.1 < a10_c / a10_s < 10.0                   # same order at contact and shock
    assert a10_s >= 3.0 * a10_r
    for k in (4, 6, 10):                                 # Delta*_5, _7, _11 small
        assert np.abs(ds[k]).max() < 0.25 * max(peak, np.abs(d10).max())
    for k in (5, 9):                                     # back to equilibrium away from the waves
        assert np.abs(ds[k][quiet]).max() < 0.05 * np.abs(ds[k]).max()


def test_sec5_delta_star_parity_with_oracle(orc, lbm):
    p = wl.shock_heavy_light(steps=2000)
    s = lbm.Solver.from_problem(p)
    s.init(*p.fields())
    s.step(p.steps)
    g = s.moments_central()
    s.close()
    O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, p.limiter, p.bc)
    O.init(*p.fields())
    O.step(p.steps)
    r = O.moments_central()
    assert np.abs(g - r).max() <= 1e-9 * np.abs(r[4:]).max()
