"""Small deviations in the float32 deviation mode (the storage g = f - f^eq0).

An isobaric thermal wave of amplitude A = 1e-5 about (rho, u, T) = (1, 0, 1), on a
periodic 128 x 4 grid with the energy-flux correction active (Pr = 0.5). After 200 steps
the float32 run's temperature deviation T - 1 matches the float64 oracle's to 1e-4 of A,
and so do its density deviation and its induced velocity. Storing f itself in float32
would round T at about 6e-8 absolute, 6e-3 of A; the deviation storage keeps the
wave's digits. The temperature is recovered in float32 from the deviation sums,
dP = (de - |j|^2/rho)/b.
"""
import numpy as np
import pytest

from paper_1305_4736_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

A = 1e-5


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1305_4736_gb300 import build, lbm as L
    build.build()
    L.load()
    return L


def _wave(nx=128, ny=4):
    x = (np.arange(nx) + 0.5) / nx
    T = np.tile(1.0 + A * np.sin(2 * np.pi * x), (ny, 1))
    rho = 1.0 / T                                       # isobaric: P = rho T = 1
    zero = np.zeros((ny, nx))
    s = wl.rates(200.0, 100.0, 400.0)                   # Pr = s8 / s5 = 0.5
    return wl.Problem("thermal_wave_1e-5", nx, ny, 1.0 / nx, 2e-4, 1.4, 0.5, s, wl.periodic_bc(),
                      rho, zero, zero.copy(), T, 200)


def test_fp32_keeps_the_digits_of_a_small_thermal_wave(orc, lbm):
    p = _wave()
    s = lbm.Solver(p.nx, p.ny, p.dx, p.dt, p.gamma, p.Pr, p.s, p.limiter, p.bc, precision=lbm.LBM_FP32_DEV)
    s.init(*p.fields())
    s.step(p.steps)
    rho, u, v, T = s.moments()
    s.close()
    O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, p.limiter, p.bc)
    O.init(*p.fields())
    O.step(p.steps)
    ro, uo, vo, To = O.moments()
    amp_T = np.abs(To - 1.0).max()
    assert 0.1 * A < amp_T < A                         # the wave has decayed but is still there
    assert np.abs((T - 1.0) - (To - 1.0)).max() <= 1e-4 * A
    assert np.abs(rho - ro).max() <= 1e-4 * A
    assert np.abs(u - uo).max() <= 1e-4 * A and np.abs(v - vo).max() <= 1e-4 * A
