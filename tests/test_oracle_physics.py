"""Physics pins of the oracle against exact solutions and closed forms (CPU only).

- the paper's discontinuity test (Sec. IV.A): a Mach-sqrt2 shock (gamma = 2)
  translating at speed 2; L1 error halves as dx halves;
- the Sod shock tube against the exact Riemann solution: L1 errors of rho, u,
  T fall monotonically under refinement (dt proportional to dx);
- shear-wave decay at nu = R T / s5 and the Chapman-Enskog value of Delta_7
  (Sec. II transport coefficients; Sec. V non-equilibrium moments);
- an isobaric thermal wave against the full linearised Navier-Stokes
  evolution with mu = rho R T/s5, mu_B = (2/3 - 2/b) mu, lambda = (b/2+1) R
  rho R T / s8 (Sec. II);
- thermal Couette flow (Sec. IV.C): the linear velocity profile and the
  viscous-heating profile, whose amplitude scales with Pr = s8/s5 only because
  of the energy-flux correction of the collision (with it the heating ratio
  Pr = 2 : Pr = 0.5 is 4; without it 1; with the opposite sign about 0); the
  deviation of the forward-Euler step is first order in dt, and its Richardson
  extrapolation meets the analytic profile.

Tolerances are set by the physics at CPU-affordable parameters and stated
next to each check.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import riemann
from oracle.analytic import couette_profile, normal_shock
from paper_1305_4736_gb300 import workloads as wl


def _run(orc, p):
    O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, p.limiter, p.bc)
    O.init(*p.fields())
    O.step(p.steps)
    return O


def test_paper_discontinuity_shock_translates_and_converges(orc):
    """gamma = 2, (1.5, 2/3, 0, 14/9) | (1, 0, 0, 1), dt = 1e-5, s5-7 = 5e4, others 1e5,
    equilibrium x ends, t = 0.06 (Sec. IV.A); exact: a shock moving at 2."""
    r2, u2, p2, S = normal_shock(1.0, 1.0, math.sqrt(2.0), 2.0)
    l1 = []
    for dx in (4e-3, 2e-3, 1e-3):
        nx = int(round(1.0 / dx))
        p = wl.riemann(nx, 1, (r2, u2, 0.0, p2 / r2), (1.0, 0.0, 0.0, 1.0), 2.0,
                       wl.rates(5e4, 5e4, 1e5), dt=1e-5, t_end=0.06, bc_kind=wl.BC_EQUILIBRIUM)
        rho = _run(orc, p).moments()[0][0]
        x = (np.arange(nx) + 0.5) * dx
        xs = 0.5 + S * p.steps * p.dt
        l1.append(np.abs(rho - np.where(x < xs, r2, 1.0)).sum() * dx)
        # the discrete shock sits where rho crosses the mid value, within two cells
        cross = x[np.argmax(rho < 0.5 * (r2 + 1.0))]
        assert abs(cross - xs) <= 2 * dx
        assert np.abs(rho[x > xs + 0.05] - 1.0).max() <= 1e-12        # undisturbed gas ahead
    assert l1[0] > l1[1] > l1[2]
    assert l1[1] / l1[2] > 1.7 and l1[0] / l1[1] > 1.7                 # first order at a shock
    assert l1[2] <= 6e-4


def test_sod_converges_to_exact_riemann_solution(orc):
    sol = riemann.solve((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
    errs = []
    for nx in (100, 200, 400):         # s dt = 0.5 at 200 cells; 50 cells would give s dt = 2
        p = wl.sod(nx, 1)
        rho, ux, _, T = (a[0] for a in _run(orc, p).moments())
        x = (np.arange(nx) + 0.5) / nx
        t = p.steps * p.dt
        re, ue, pe = sol.sample((x - 0.5) / t)
        errs.append([np.abs(rho - re).mean(), np.abs(ux - ue).mean(), np.abs(T - pe / re).mean()])
    errs = np.array(errs)
    assert np.all(np.diff(errs, axis=0) < 0), errs
    assert errs[1, 0] <= 5e-3        # L1(rho) at the 200-cell configuration: 4.55e-3 recorded


def test_shear_wave_decay_and_delta7(orc):
    nx, s5, dt, A = 64, 50.0, 1e-4, 1e-3
    x = (np.arange(nx) + 0.5) / nx
    k = 2 * math.pi
    O = orc.Oracle(nx, 1, 1.0 / nx, dt, 1.4, wl.rates(s5), 0, wl.periodic_bc())
    O.init(1.0, 0.0, A * np.sin(k * x)[None, :], 1.0)
    ts, amps, d7 = [], [], []
    for j in range(5):
        O.step(1000)
        rho, ux, uy, T, D = O.moments(delta=True)
        a = 2 * np.mean(uy[0] * np.sin(k * x))
        ts.append((j + 1) * 1000 * dt)
        amps.append(a)
        ce = -(rho[0] * T[0] / s5) * k * a * np.cos(k * x)          # -(P/s7)(d_x u_y + d_y u_x)
        d7.append(np.sum(D[6, 0] * ce) / np.sum(ce * ce))
    rate = -np.polyfit(ts, np.log(amps), 1)[0]
    assert rate / (k * k / s5) == pytest.approx(1.0, abs=0.01)        # nu = R T / s5
    assert d7[-1] == pytest.approx(1.0, abs=0.01)


def _ns_matrix(k, s5, s8, b):
    """Linearised NS (rho0 = T0 = 1, R = 1) for (d rho, d u, d T) ~ exp(i k x)."""
    mu_long = (2.0 - 2.0 / b) / s5            # 2 mu - 2/3 mu + mu_B
    lam = (b / 2.0 + 1.0) / s8
    cv = b / 2.0
    return np.array([[0, -1j * k, 0], [-1j * k, -mu_long * k * k, -1j * k],
                     [0, -1j * k / cv, -lam * k * k / cv]], dtype=complex)


@pytest.mark.parametrize("s5,s8", [(300.0, 150.0), (150.0, 300.0)])
def test_thermal_wave_follows_linearised_navier_stokes(orc, s5, s8):
    nx, dt, A, gamma = 64, 5e-5, 1e-4, 1.4
    b = 2.0 / (gamma - 1.0)
    k = 2 * math.pi
    x = (np.arange(nx) + 0.5) / nx
    T0 = 1.0 + A * np.cos(k * x)[None, :]
    O = orc.Oracle(nx, 1, 1.0 / nx, dt, gamma, wl.rates(s5, s8, 600.0), 0, wl.periodic_bc())
    O.init(1.0 / T0, 0.0, 0.0, T0)                                   # isobaric
    c = lambda a: 2 * np.mean((a[0] - a[0].mean()) * np.cos(k * x))  # noqa: E731
    sn = lambda a: 2 * np.mean((a[0] - a[0].mean()) * np.sin(k * x))  # noqa: E731
    rho, ux, uy, T = O.moments()
    x0 = np.array([c(rho), 0.0, c(T)], dtype=complex)
    Mx = _ns_matrix(k, s5, s8, b)
    worst = 0.0
    for j in range(10):
        O.step(2000)
        rho, ux, uy, T = O.moments()
        xe = expm(Mx * (j + 1) * 2000 * dt) @ x0
        worst = max(worst, np.abs([c(rho) - xe[0].real, sn(ux) + xe[1].imag, c(T) - xe[2].real]).max())
    assert worst <= 0.015 * A        # 0.45% of A measured; lambda off by 2x gives ~20%


def _couette_run(args):
    """Thermal Couette run from the analytic profile to steady state (spawned worker)."""
    Pr, dt, ny, s5, efolds = args
    from oracle import oracle as o
    from oracle.analytic import couette_profile
    from paper_1305_4736_gb300 import workloads as w
    o.load()
    o.set_threads(1)
    u0, gamma = 0.2, 1.4
    b = 2.0 / (gamma - 1.0)
    y = (np.arange(ny) + 0.5) / ny
    p = w.couette(Pr, nx=1, ny=ny, dt=dt, s5=s5, gamma=gamma, u0=u0)
    ue, Te = couette_profile(y, u0, Pr, b)
    O = o.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, o.LIM_LW, p.bc)
    O.init(1.0, ue[:, None], 0.0, Te[:, None])
    slowest = min(1.0 / s5, (b / 2.0 + 1.0) / (b / 2.0) / (Pr * s5))     # nu, thermal diffusivity
    n = int(round(efolds / (math.pi ** 2 * slowest) / dt / 1000.0)) * 1000
    O.step(n - 1000)
    T_prev = O.moments()[3][:, 0]
    O.step(1000)
    rho, ux, uy, T = (a[:, 0] for a in O.moments())
    return ux, T, float(np.abs(T - T_prev).max())


def test_couette_profiles_and_prandtl_scaling():
    """Sec. IV.C: walls at y = 0 (rest) and y = 1 (u0 = 0.2), T_w = 1, gamma = 1.4, s5 = others
    = 400, s8 = Pr s5, 50 cells (dx = 0.02), Lax-Wendroff limiter, started from the analytic profile and run
    for 7 e-folds of the slowest diffusion mode (max |dT| per 1000 steps then below 1e-9).

    The forward-Euler step (Sec. III) is first order in time, and on this problem its error is
    first order in s dt: at s5 dt = 0.2 the heating is 13% low at Pr = 2, at 0.1 it is 7% low
    (ratio 2).  The grid does not matter (40, 50, 80 and 160 cells give the same deviation), and
    the Knudsen effect is below 0.5% at s5 = 400.  So the test checks the first-order time error,
    then the Richardson extrapolation 2 T(dt/2) - T(dt) against the analytic profile: the linear
    velocity to 1e-4 u0 and the temperature to 2% of the mid-channel heating (pin P11), and the
    Prandtl scaling of the heating (ratio 4 between Pr = 2 and Pr = 0.5) to 3%; that scaling
    exists only through the energy-flux correction of the collision.
    (The monotonised-central limiter on the same grid stays 7-16% off for any dt: it clips to
    first order where the y-moving populations have their extrema; see the design notes.)"""
    import multiprocessing as mp
    from oracle.analytic import couette_profile
    ny, s5, u0 = 50, 400.0, 0.2
    b = 5.0
    y = (np.arange(ny) + 0.5) / ny
    cases = [(Pr, sdt / s5, ny, s5, 7.0) for Pr in (0.5, 2.0) for sdt in (0.2, 0.1)]
    with mp.get_context("spawn").Pool(4) as pool:
        runs = pool.map(_couette_run, cases)
    heat = {}
    for k, Pr in enumerate((0.5, 2.0)):
        (ux1, T1, d1), (ux2, T2, d2) = runs[2 * k], runs[2 * k + 1]
        ue, Te = couette_profile(y, u0, Pr, b)
        mid = Pr * u0 * u0 / (4.0 * (b + 2.0))
        assert d1 < 1e-9 and d2 < 1e-9                                  # steady
        assert np.abs(ux1 - ue).max() <= 1e-4 * u0 and np.abs(ux2 - ue).max() <= 1e-4 * u0
        X = np.stack([y * (1 - y), np.ones_like(y)], 1)
        c1, c2 = (np.linalg.lstsq(X, T - 1.0, rcond=None)[0][0] / (4.0 * mid) for T in (T1, T2))
        assert 1.6 <= (c1 - 1.0) / (c2 - 1.0) <= 2.4, (Pr, c1, c2)        # heating error first order in dt
        TR = 2.0 * T2 - T1
        assert np.abs(TR - Te).max() <= 0.02 * mid, (Pr, np.abs(TR - Te).max() / mid)
        heat[Pr] = np.linalg.lstsq(X, TR - 1.0, rcond=None)[0][0]
    assert heat[2.0] / heat[0.5] == pytest.approx(4.0, rel=0.03)       # 1.6% measured: the O((s dt)^2) remainder at Pr = 2
