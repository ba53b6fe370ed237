"""Pins of the oracle's time step against properties the paper's scheme fixes (CPU only).

- a uniform equilibrium state is stationary under every boundary kind;
- on a doubly periodic grid the flux form telescopes: each population's sum is
  invariant when s = 0, and mass, momentum and energy are invariant for any s;
- Courant number 1 turns the limited update of an axis population into an
  exact one-cell shift (Sec. III: the flux correction carries 1 - c);
- psi = 1 and psi = 0 are the textbook Lax-Wendroff and first-order upwind
  updates of linear advection (Sec. III), and the MC limiter keeps a
  monotone profile monotone (no new extrema, total variation not increased);
- 90-degree rotation and mirror images of the data give the rotated /
  mirrored result (the velocity set is invariant under both).
"""
import math

import numpy as np
import pytest

from paper_1305_4736_gb300 import workloads as wl

BC = wl


def _mk(orc, nx, ny, dx, dt, gamma, s, limiter=0, bc=None):
    return orc.Oracle(nx, ny, dx, dt, gamma, s, limiter, bc if bc is not None else wl.periodic_bc())


@pytest.mark.parametrize("kind", [BC.BC_PERIODIC, BC.BC_ZERO_GRADIENT, BC.BC_EQUILIBRIUM, BC.BC_NEQ_WALL])
def test_uniform_state_is_stationary(orc, kind):
    rho, ux, uy, T = 1.3, 0.1, -0.05, 0.9
    edge = (kind, rho, ux, uy, T)
    bc = [edge] * 4
    O = _mk(orc, 6, 5, 0.01, 1e-4, 1.4, wl.rates(1e3, 600.0, 2e3), 0, bc)
    O.init(rho, ux, uy, T)
    f0 = O.get_state()
    O.step(1000)
    f1 = O.get_state()
    assert np.abs(f1 - f0).max() <= 1e-13 * np.abs(f0).max()


def _smooth_fields(nx, ny, seed, amp=0.05):
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    out = []
    for base in (1.0, 0.0, 0.0, 1.0):
        a, b, p, q = rng.uniform(-1, 1, 4)
        out.append(base + amp * (a * np.sin(2 * math.pi * X + p) + b * np.cos(2 * math.pi * Y + q)))
    return out


def test_periodic_totals_are_invariant(orc):
    nx, ny = 16, 12
    O = _mk(orc, nx, ny, 1.0 / nx, 2e-3, 1.4, wl.rates(200.0, 100.0, 300.0))
    O.init(*_smooth_fields(nx, ny, 1))
    t0 = O.totals()
    O.step(200)
    t1 = O.totals()
    scale = np.abs(t0).max()
    assert np.abs(t1 - t0).max() <= 1e-13 * scale


def test_periodic_population_sums_invariant_without_collision(orc):
    nx, ny = 16, 12
    O = _mk(orc, nx, ny, 1.0 / nx, 1e-3, 1.4, np.zeros(16))
    O.init(*_smooth_fields(nx, ny, 2, amp=0.2))
    s0 = O.get_state().sum(axis=(1, 2))
    O.step(100)
    s1 = O.get_state().sum(axis=(1, 2))
    assert np.abs(s1 - s0).max() <= 1e-13 * np.abs(s0).max()


@pytest.mark.parametrize("shell", [0, 1])
@pytest.mark.parametrize("limiter", [0, 1, 2])
def test_courant_one_is_exact_shift_for_axis_shells(orc, shell, limiter):
    """With s = 0 and c = |v| dt/dx = 1 an axis population moves one cell per step, bit for bit."""
    A = (1.0, 1.0 / 6.0)[shell]
    nx, ny = 9, 7
    O = _mk(orc, nx, ny, 1.0, A, 1.4, np.zeros(16), limiter)
    rng = np.random.default_rng(3)
    f = np.zeros((16, ny, nx))
    f[4 * shell:4 * shell + 4] = rng.uniform(1.0, 2.0, (4, ny, nx))   # Sterbenz range: exact differences
    O.set_state(f)
    O.step(3)
    g = O.get_state()
    shifts = [(1, 0), (0, 1), (-1, 0), (0, -1)]
    for k, (sx, sy) in enumerate(shifts):
        q = 4 * shell + k
        expect = np.roll(np.roll(f[q], 3 * sx, axis=1), 3 * sy, axis=0)
        assert np.array_equal(g[q], expect)


@pytest.mark.parametrize("shell", [2, 3])
def test_courant_one_diagonal_projection(orc, shell):
    """At c = 1 the unsplit projection of a diagonal population gives
    f(J - sx) + f(J - sy) - f(J) (both projections taken from f^n)."""
    A = (1.0 / math.sqrt(2.0), math.sqrt(2.0) / 3.0)[shell - 2]
    nx, ny = 8, 6
    O = _mk(orc, nx, ny, 1.0, A, 1.4, np.zeros(16), 0)
    rng = np.random.default_rng(4)
    f = np.zeros((16, ny, nx))
    f[4 * shell:4 * shell + 4] = rng.uniform(1.0, 2.0, (4, ny, nx))
    O.set_state(f)
    O.step(1)
    g = O.get_state()
    signs = [(1, 1), (-1, 1), (-1, -1), (1, -1)]
    for k, (sx, sy) in enumerate(signs):
        q = 4 * shell + k
        expect = np.roll(f[q], sx, axis=1) + np.roll(f[q], sy, axis=0) - f[q]
        assert np.abs(g[q] - expect).max() <= 4e-15 * np.abs(f[q]).max()


def _advect_1d(orc, limiter, c, q, profile):
    nx = profile.size
    O = _mk(orc, nx, 1, 1.0, c, 1.4, np.zeros(16), limiter)   # dx = 1, dt = c: axis shell 1
    f = np.zeros((16, 1, nx))
    f[q, 0] = profile
    O.set_state(f)
    O.step(1)
    return O.get_state()[q, 0]


@pytest.mark.parametrize("q,sign", [(0, 1), (2, -1)])
def test_lax_wendroff_and_upwind_special_cases(orc, q, sign):
    rng = np.random.default_rng(5)
    u = rng.uniform(0.5, 1.5, 40)
    c = 0.37
    up = np.roll(u, sign)       # u_{j - sigma}
    dn = np.roll(u, -sign)      # u_{j + sigma}
    lw = u - 0.5 * c * (dn - up) + 0.5 * c * c * (dn - 2 * u + up)
    uw = u - c * (u - up)
    assert np.abs(_advect_1d(orc, 1, c, q, u) - lw).max() <= 1e-15 * 4
    assert np.abs(_advect_1d(orc, 2, c, q, u) - uw).max() <= 1e-15 * 4


def test_mc_limiter_is_tvd_on_a_step(orc):
    nx = 60
    u = np.where(np.arange(nx) < 20, 2.0, 1.0) + np.where(np.arange(nx) >= 45, 0.5, 0.0)
    O = _mk(orc, nx, 1, 1.0, 0.45, 1.4, np.zeros(16), 0)
    f = np.zeros((16, 1, nx))
    f[0, 0] = u
    O.set_state(f)
    tv0 = np.abs(np.diff(np.r_[u, u[0]])).sum()
    for _ in range(40):
        O.step(1)
        g = O.get_state()[0, 0]
        assert g.min() >= u.min() - 1e-14 and g.max() <= u.max() + 1e-14
        assert np.abs(np.diff(np.r_[g, g[0]])).sum() <= tv0 + 1e-12


def _run_fields(orc, fields, n, steps, s):
    O = _mk(orc, n, n, 1.0 / n, 1e-3, 1.4, s)
    O.init(*fields)
    O.step(steps)
    return O.moments()


def test_rotation_by_90_degrees(orc):
    n = 12
    rho, ux, uy, T = _smooth_fields(n, n, 6, amp=0.1)
    s = wl.rates(300.0, 150.0, 400.0)
    rot = lambda a: a.T[:, ::-1]  # noqa: E731  (i, j) -> (n-1-j, i): counter-clockwise
    a = _run_fields(orc, (rho, ux, uy, T), n, 20, s)
    b = _run_fields(orc, (rot(rho), rot(-uy), rot(ux), rot(T)), n, 20, s)
    exp = (rot(a[0]), rot(-a[2]), rot(a[1]), rot(a[3]))
    for got, want in zip(b, exp):
        assert np.abs(got - want).max() <= 1e-13


def test_mirror_in_x(orc):
    n = 12
    rho, ux, uy, T = _smooth_fields(n, n, 7, amp=0.1)
    s = wl.rates(300.0, 150.0, 400.0)
    mir = lambda a: a[:, ::-1]  # noqa: E731
    a = _run_fields(orc, (rho, ux, uy, T), n, 20, s)
    b = _run_fields(orc, (mir(rho), -mir(ux), mir(uy), mir(T)), n, 20, s)
    exp = (mir(a[0]), -mir(a[1]), mir(a[2]), mir(a[3]))
    for got, want in zip(b, exp):
        assert np.abs(got - want).max() <= 1e-13
