"""Thermal Couette flow run to steady state on the GPU against the analytic profile (Sec. IV.C).

4 x 50 cells (dx = 0.02), periodic x, non-equilibrium extrapolation walls at y = 0 (rest) and
y = 1 (u0 = 0.2), T_w = 1, gamma = 1.4, s5 = others = 400, s8 = Pr s5 for Pr = 0.5, 1, 2, the
Lax-Wendroff limiter; started from the analytic profile and stepped (FP64, one batch of all six
runs); each run's profile is taken when its max |dT| over 1000 steps first falls below 1e-9.

The forward-Euler step is first order in time and on this flow its error is first order in
s dt (grid independent, measured with the oracle on 40 to 160 cells), so each Pr runs at
s5 dt = 0.2 and 0.1 (dt = 5e-4, 2.5e-4): the heating error must halve with dt, and the Richardson
extrapolation 2 T(dt/2) - T(dt) must meet the analytic profile within 2% of the mid-channel
heating, the velocity within 1e-4 u0 (pin P11), and the heating must scale with Pr (ratio 4
between Pr = 2 and Pr = 0.5, to 3%).  The oracle checks the same flow on the CPU
(tests/test_oracle_physics.py); parity of the GPU path with the oracle over the first 1000 steps
of this configuration family is in tests/test_gpu_parity.py.
"""
import numpy as np
import pytest

from oracle.analytic import couette_profile
from paper_1305_4736_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_couette_converges_to_the_analytic_profile():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1305_4736_gb300 import build, lbm
    build.build()
    lbm.load()
    nx, ny, s5, u0, gamma = 4, 50, 400.0, 0.2, 1.4
    b = 2.0 / (gamma - 1.0)
    y = (np.arange(ny) + 0.5) / ny
    cases = [(Pr, sdt / s5) for Pr in (0.5, 1.0, 2.0) for sdt in (0.2, 0.1)]
    solvers = []
    for Pr, dt in cases:
        p = wl.couette(Pr, nx=nx, ny=ny, dt=dt, s5=s5, gamma=gamma, u0=u0)
        p.limiter = lbm.LBM_LIMITER_LW
        ue, Te = couette_profile(y, u0, Pr, b)
        s = lbm.Solver.from_problem(p)
        s.init(np.ones((ny, nx)), np.repeat(ue[:, None], nx, 1), np.zeros((ny, nx)), np.repeat(Te[:, None], nx, 1))
        solvers.append(s)
    batch = lbm.Batch(solvers)
    steps = 0
    fields = [None] * len(solvers)          # each run's moments when it first meets the criterion
    while any(f is None for f in fields):
        assert steps < 4_000_000, f"no steady state after {steps} steps"
        batch.step(20000)
        before = [s.moments()[3] for s in solvers]
        batch.step(1000)
        steps += 21000
        for k, s in enumerate(solvers):
            m = s.moments()
            if fields[k] is None and float(np.abs(m[3] - before[k]).max()) < 1e-9:
                fields[k] = m
    batch.close()
    for s in solvers:
        s.close()
    X = np.stack([y * (1 - y), np.ones_like(y)], 1)
    heat = {}
    for k, Pr in enumerate((0.5, 1.0, 2.0)):
        ue, Te = couette_profile(y, u0, Pr, b)
        mid = Pr * u0 * u0 / (4.0 * (b + 2.0))
        (_, ux1, _, T1), (_, ux2, _, T2) = fields[2 * k], fields[2 * k + 1]
        assert np.abs(T1 - T1[:, :1]).max() <= 1e-12 and np.abs(T2 - T2[:, :1]).max() <= 1e-12   # uniform in x
        T1, T2, ux1, ux2 = T1[:, 0], T2[:, 0], ux1[:, 0], ux2[:, 0]
        assert np.abs(ux1 - ue).max() <= 1e-4 * u0 and np.abs(ux2 - ue).max() <= 1e-4 * u0
        c1, c2 = (np.linalg.lstsq(X, T - 1.0, rcond=None)[0][0] / (4.0 * mid) for T in (T1, T2))
        assert 1.6 <= (c1 - 1.0) / (c2 - 1.0) <= 2.4, (Pr, c1, c2)       # heating error first order in dt
        TR = 2.0 * T2 - T1
        err = np.abs(TR - Te).max() / mid
        assert err <= 0.02, (Pr, err)
        heat[Pr] = np.linalg.lstsq(X, TR - 1.0, rcond=None)[0][0]
    assert heat[2.0] / heat[0.5] == pytest.approx(4.0, rel=0.03)       # 1.6% measured: the O((s dt)^2) remainder at Pr = 2
