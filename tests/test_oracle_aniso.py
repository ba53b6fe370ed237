"""Pins of the oracle on grids with dy != dx (CPU only).

The update of Sec. III projects the convection on each axis with that axis's
Courant number |v_i,alpha| dt / d_alpha, and the central differences of the
energy-flux correction (Sec. II) divide by 2 d_alpha.  Three properties fix the
roles of dx and dy:
- a 90-degree rotation of the data, with dx and dy exchanged, gives the rotated
  result (a wrong spacing in either the Courant numbers or the gradients of the
  correction breaks it, since the correction is active at Pr != 1);
- a state that is uniform along y evolves independently of dy, bit for bit (no
  y difference, no y gradient), and likewise along x;
- at |v_y| dt / dy = 1 a y-moving population of an axis shell moves exactly one
  row per step, whatever dx is.
"""
import numpy as np
import pytest

from paper_1305_4736_gb300 import workloads as wl


def _smooth(nx, ny, seed, amp):
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    out = []
    for base in (1.0, 0.0, 0.0, 1.0):
        a = rng.uniform(-1, 1, 3)
        p = rng.uniform(0, 2 * np.pi, 3)
        f = (a[0] * np.sin(2 * np.pi * X + p[0]) + a[1] * np.sin(2 * np.pi * Y + p[1])
             + a[2] * np.sin(2 * np.pi * (X + Y) + p[2]))
        out.append(base + amp * f)
    return out


def _run(orc, fields, nx, ny, dx, dy, steps, s, dt=2e-4):
    O = orc.Oracle(nx, ny, dx, dt, 1.4, s, 0, wl.periodic_bc(), dy=dy)
    O.init(*fields)
    O.step(steps)
    return O.moments()


def test_rotation_exchanges_dx_and_dy(orc):
    nx, ny, dx, dy = 14, 10, 1.0 / 14, 1.0 / 25
    rho, ux, uy, T = _smooth(nx, ny, 11, amp=0.1)
    s = wl.rates(300.0, 150.0, 400.0)                  # Pr = 0.5: the gradient correction is on
    rot = lambda a: a.T[:, ::-1]  # noqa: E731  counter-clockwise: new x = old y
    a = _run(orc, (rho, ux, uy, T), nx, ny, dx, dy, 20, s)
    b = _run(orc, (rot(rho), rot(-uy), rot(ux), rot(T)), ny, nx, dy, dx, 20, s)
    exp = (rot(a[0]), rot(-a[2]), rot(a[1]), rot(a[3]))
    for got, want in zip(b, exp):
        assert np.abs(got - want).max() <= 1e-13
    # and the spacing matters: the same data on the unrotated spacings differ
    c = _run(orc, (rot(rho), rot(-uy), rot(ux), rot(T)), ny, nx, dx, dy, 20, s)
    assert np.abs(c[3] - b[3]).max() > 1e-9


@pytest.mark.parametrize("axis", ["x", "y"])
def test_uniform_direction_ignores_its_spacing(orc, axis):
    n = 16
    x = (np.arange(n) + 0.5) / n
    prof = [1.0 + 0.1 * np.sin(2 * np.pi * x), 0.05 * np.cos(2 * np.pi * x), 0.02 * np.sin(4 * np.pi * x),
            1.0 + 0.05 * np.cos(2 * np.pi * x)]
    if axis == "x":       # varies along x, uniform along y: dy must not matter
        fields = [np.tile(p, (4, 1)) for p in prof]
        nx, ny = n, 4
        runs = [_run(orc, fields, nx, ny, 1.0 / n, dy, 30, wl.rates(300.0, 150.0, 400.0))
                for dy in (1.0 / n, 0.5 / n, 3.0 / n)]
    else:                 # varies along y, uniform along x: dx must not matter
        fields = [np.tile(p[:, None], (1, 4)) for p in prof]
        nx, ny = 4, n
        runs = [_run(orc, fields, nx, ny, dx, 1.0 / n, 30, wl.rates(300.0, 150.0, 400.0))
                for dx in (1.0 / n, 0.5 / n, 3.0 / n)]
    for r in runs[1:]:
        for a, b in zip(r, runs[0]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("shell", [0, 1])
def test_courant_one_in_y_is_exact_row_shift(orc, shell):
    A = (1.0, 1.0 / 6.0)[shell]
    nx, ny = 7, 9
    dy = 1.0
    O = orc.Oracle(nx, ny, 2.0 * dy, A * dy, 1.4, np.zeros(16), 0, wl.periodic_bc(), dy=dy)
    rng = np.random.default_rng(6)
    f = np.zeros((16, ny, nx))
    f[4 * shell:4 * shell + 4] = rng.uniform(1.0, 2.0, (4, ny, nx))
    O.set_state(f)
    O.step(3)
    g = O.get_state()
    for k, sy in ((1, 1), (3, -1)):              # the y-moving populations of the shell
        q = 4 * shell + k
        assert np.array_equal(g[q], np.roll(f[q], 3 * sy, axis=0))
