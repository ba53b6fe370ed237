"""GPU parity of the double-float float64 kernel (lbm_options.step_kernel = 8, and 9 on narrow
32 x 4 tiles).

The populations stay float64; the step's arithmetic runs in double-float form on the float32
pipe (about 2^-47 rounding per operation instead of 2^-53).  The bar is the float64 mode's:
max relative error <= 1e-10 on rho, u, T against the oracle (u as a vector), here also on the
populations themselves, for every limiter, with walls and the energy-flux correction active
(Pr != 1), with dy != dx, on ragged tiles, after 1000 steps of the reduced shock-interface
and shear-layer configurations, and at full size (8192^2, sampled cells recomputed by the
oracle from the GPU's previous step).  Against the float64 tile kernel it agrees to a few
parts in 1e13 after 60 steps.
"""
import numpy as np
import pytest

from _gpu_helpers import fp64_errors
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


def _run(lbm, p, steps, kernel=8, limiter=None):
    s = lbm.Solver(p.nx, p.ny, p.dx, p.dt, p.gamma, p.Pr, p.s, p.limiter if limiter is None else limiter, p.bc,
                   step_kernel=kernel, dy=p.dy)
    assert s.step_kernel == kernel
    s.init(*p.fields())
    if steps:
        s.step(steps)
    return s


def _oracle(orc, p, steps, limiter=None):
    O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, p.limiter if limiter is None else limiter, p.bc, dy=p.dy)
    O.init(*p.fields())
    O.step(steps)
    return O


def _check(s, O):
    errs = fp64_errors(s, O)
    for k, v in errs.items():
        assert v <= TOL, f"{k}: {v:.3e} ({errs})"
    fo = O.get_state()
    assert np.abs(s.get_state() - fo).max() <= TOL * np.abs(fo).max()


@pytest.mark.parametrize("limiter", [0, 1, 2])
def test_dd_kernel_each_limiter_against_oracle(orc, lbm, limiter):
    p = wl.shock_interface(nx=150, ny=70, steps=120)          # ragged against 32 x 32 tiles
    _check(_run(lbm, p, 120, limiter=limiter), _oracle(orc, p, 120, limiter))


def test_dd_kernel_walls_and_energy_flux_correction(orc, lbm):
    """NEQ walls on x (moving, heated), equilibrium and zero-gradient y edges, Pr = 0.71."""
    p = wl.shear_layer(96, ny=66)
    p.bc = [(wl.BC_NEQ_WALL, 1.0, 0.0, 0.02, 1.01), (wl.BC_NEQ_WALL, 1.0, 0.0, -0.03, 0.99),
            (wl.BC_EQUILIBRIUM, 1.02, 0.01, 0.0, 1.0), (wl.BC_ZERO_GRADIENT, 0, 0, 0, 0)]
    _check(_run(lbm, p, 300), _oracle(orc, p, 300))


@pytest.mark.parametrize("Pr", [0.5, 2.0])
def test_dd_kernel_couette_1000_steps(orc, lbm, Pr):
    p = wl.couette(Pr, nx=32, ny=200)
    _check(_run(lbm, p, 1000), _oracle(orc, p, 1000))


@pytest.mark.parametrize("ratio", [0.7, 1.6])
def test_dd_kernel_dy_not_dx(orc, lbm, ratio):
    p = wl.shear_layer(100, ny=70)
    p.dy = ratio * p.dx
    _check(_run(lbm, p, 200), _oracle(orc, p, 200))


def test_dd_kernel_periodic_x_wrap(lbm):
    """A grid large enough for the in-kernel x wrap of periodic edge tiles (ghost launch copies
    only the ghost rows), against the float64 tile kernel after 20 steps."""
    p = wl.shear_layer(3000, ny=3500)
    s = _run(lbm, p, 20)
    t = _run(lbm, p, 20, kernel=2)
    a, b = s.get_state_rows(0, p.ny), t.get_state_rows(0, p.ny)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("limiter", [0, 1, 2])
def test_dd_kernel_matches_float64_tile_kernel(lbm, limiter):
    p = wl.shock_interface(nx=150, ny=70, steps=60)
    a = _run(lbm, p, 60, kernel=8, limiter=limiter).get_state()
    b = _run(lbm, p, 60, kernel=2, limiter=limiter).get_state()
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("name", ["shock_interface_512x128", "shear_layer_1024x1024"])
def test_dd_kernel_reduced_configs_1000_steps(orc, lbm, name):
    p = (wl.shock_interface(nx=512, ny=128, steps=1000) if name.startswith("shock")
         else wl.shear_layer(1024, steps=1000))
    s = _run(lbm, p, 1000)
    O = _oracle(orc, p, 1000)
    errs = fp64_errors(s, O)
    for k, v in errs.items():
        assert v <= TOL, f"{k}: {v:.3e} ({errs})"


@pytest.mark.parametrize("nx,ny,want", [(512, 512, 8), (384, 384, 8), (8192, 32, 8), (256, 256, 9), (33, 32, 9),
                                         (33, 31, 9), (200, 4, 9), (2048, 16, 9), (31, 64, 7), (4, 200, 7),
                                         (200, 3, 7)])
def test_automatic_float64_choice(lbm, nx, ny, want):
    """The automatic float64 choice is the double-float kernel: on 32 x 32 tiles where the grid
    has at least two thirds of a wave of them (101 on 152 SMs), else on 32 x 4 tiles where those
    fit (32 columns, 4 rows); grids narrower than that keep the float64-pipe kernels."""
    p = wl.shear_layer(max(nx, ny), ny=ny)
    p.nx = nx
    p.rho, p.ux, p.uy, p.T = (np.ascontiguousarray(a[:, :nx]) for a in (p.rho, p.ux, p.uy, p.T))
    s = lbm.Solver.from_problem(p)
    assert s.step_kernel == want
    s.close()


def test_dd_kernel_rejected_in_fp32_mode(lbm):
    p = wl.shear_layer(64, ny=32)
    with pytest.raises(lbm.LbmError):
        lbm.Solver.from_problem(p, precision=1, step_kernel=8)


def test_dd_kernel_autotune_candidate(lbm):
    p = wl.shear_layer(512, ny=256)
    s = lbm.Solver.from_problem(p)
    s.init(*p.fields())
    choice = s.autotune(reps=3)
    assert choice in (1, 2, 3, 4, 5, 7, 8, 9) and s.step_kernel == choice
    s.close()


def test_dd_kernel_full_size_sampled(orc, lbm):
    """8192 x 8192 shear layer in the benchmark's float64 launch configuration (the automatic
    choice is the double-float kernel): after 3 steps, 64 seeded cells of step 4 are
    recomputed by the oracle from the GPU's step-3 rows; 1e-13 of f."""
    from test_gpu_parity import _patch
    p = wl.shear_layer(8192)
    s = lbm.Solver.from_problem(p)
    assert s.step_kernel == 8
    s.init(*p.fields())
    s.step(3)
    rng = np.random.default_rng(7)
    ys = rng.integers(2, p.ny - 2, 64)
    xs = rng.integers(0, p.nx, 64)
    before = {int(y): s.get_state_rows(int(y) - 2, 5) for y in set(ys.tolist())}
    s.step(1)
    worst = 0.0
    for y, x in zip(ys.tolist(), xs.tolist()):
        want = orc.update_patch(_patch(before[y], 2, x, p.nx), p.dx, p.dt, p.gamma, p.s, p.limiter)
        got = s.get_state_rows(y, 1)[:, 0, x]
        worst = max(worst, np.abs(got - want).max() / np.abs(want).max())
    s.close()
    assert worst <= 1e-13, worst


@pytest.mark.parametrize("kernel", [8, 1])
def test_uniform_equilibrium_stays_stationary(lbm, kernel):
    """A uniform equilibrium on a doubly periodic grid (rho = 1.3, u = (0.1, -0.05), T = 0.9,
    Pr != 1) is a fixed point of the step (pin P4 of the oracle): after 1000 steps the float64
    populations are unchanged to 1e-13 of their size, with the double-float kernel's rounding
    of every value to 48 bits and back each step, as with the float64 plain kernel."""
    p = wl.shear_layer(64, ny=48)
    one = np.ones((p.ny, p.nx))
    p.rho, p.ux, p.uy, p.T = 1.3 * one, 0.1 * one, -0.05 * one, 0.9 * one
    s = _run(lbm, p, 0, kernel=kernel)
    f0 = s.get_state()
    s.step(1000)
    f1 = s.get_state()
    assert np.abs(f1 - f0).max() <= 1e-13 * np.abs(f0).max()
    s.close()


def test_dd_kernel_conserves_periodic_totals(lbm):
    """Mass, momentum and energy of a doubly periodic shear layer after 500 double-float steps
    equal the initial totals to 1e-12 of their size (the collision conserves them exactly and
    the flux form telescopes; what remains is the rounding of the float64 stores)."""
    p = wl.shear_layer(128)
    s = _run(lbm, p, 0)
    t0 = s.totals()
    s.step(500)
    t1 = s.totals()
    assert np.abs(t1 - t0).max() <= 1e-12 * np.abs(t0).max()
    s.close()


# ---- narrow tiles (step_kernel 9): grids of 4 to 31 rows ----

@pytest.mark.parametrize("limiter", [0, 1, 2])
def test_narrow_dd_kernel_each_limiter_against_oracle(orc, lbm, limiter):
    p = wl.shock_interface(nx=150, ny=13, steps=120)          # ragged against 32 x 4 tiles
    _check(_run(lbm, p, 120, kernel=9, limiter=limiter), _oracle(orc, p, 120, limiter))


def test_narrow_dd_kernel_walls_and_energy_flux_correction(orc, lbm):
    """NEQ walls on x (moving, heated), equilibrium and zero-gradient y edges, Pr = 0.71, on a
    grid of 10 rows."""
    p = wl.shear_layer(96, ny=10)
    p.bc = [(wl.BC_NEQ_WALL, 1.0, 0.0, 0.02, 1.01), (wl.BC_NEQ_WALL, 1.0, 0.0, -0.03, 0.99),
            (wl.BC_EQUILIBRIUM, 1.02, 0.01, 0.0, 1.0), (wl.BC_ZERO_GRADIENT, 0, 0, 0, 0)]
    _check(_run(lbm, p, 300, kernel=9), _oracle(orc, p, 300))


@pytest.mark.parametrize("Pr", [0.5, 2.0])
def test_narrow_dd_kernel_couette_channel(orc, lbm, Pr):
    """A 24-cell Couette channel (walls at y) on narrow tiles, 1000 steps."""
    p = wl.couette(Pr, nx=32, ny=24)
    _check(_run(lbm, p, 1000, kernel=9), _oracle(orc, p, 1000))


def test_narrow_dd_kernel_dy_not_dx(orc, lbm):
    p = wl.shear_layer(100, ny=7)
    p.dy = 1.6 * p.dx
    _check(_run(lbm, p, 200, kernel=9), _oracle(orc, p, 200))


def test_narrow_dd_kernel_sod_full_solve(orc, lbm):
    """The 200 x 4 Sod tube, automatic float64 choice (narrow tiles), the full 2000-step solve."""
    p = wl.sod(200, 4)
    s = lbm.Solver.from_problem(p)
    assert s.step_kernel == 9
    s.init(*p.fields())
    s.step(2000)
    _check(s, _oracle(orc, p, 2000))


@pytest.mark.parametrize("limiter", [0, 1, 2])
def test_narrow_dd_kernel_matches_wide_tiles_and_plain(lbm, limiter):
    """On a grid where both fit, narrow and 32 x 32 tiles give the same bits after 60 steps (the
    same double-float operations on each value; the tiles only change where a value is staged),
    and both match the float64 plain kernel to 1e-12."""
    p = wl.shock_interface(nx=150, ny=70, steps=60)
    a = _run(lbm, p, 60, kernel=9, limiter=limiter).get_state()
    b = _run(lbm, p, 60, kernel=8, limiter=limiter).get_state()
    c = _run(lbm, p, 60, kernel=1, limiter=limiter).get_state()
    assert np.array_equal(a, b)
    assert np.abs(a - c).max() <= 1e-12 * np.abs(c).max()


def test_narrow_dd_kernel_rejected_where_it_does_not_fit(lbm):
    """Narrow tiles need 32 columns and 4 rows; codes above 9 are unknown."""
    with pytest.raises(lbm.LbmError):
        lbm.Solver.from_problem(wl.shear_layer(64, ny=32), step_kernel=10)
    for nx, ny in ((31, 16), (64, 3)):
        p = wl.shear_layer(max(nx, ny), ny=ny)
        p.nx = nx
        p.rho, p.ux, p.uy, p.T = (np.ascontiguousarray(a[:, :nx]) for a in (p.rho, p.ux, p.uy, p.T))
        with pytest.raises(lbm.LbmError):
            lbm.Solver.from_problem(p, step_kernel=9)
