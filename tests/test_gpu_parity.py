"""GPU parity: the CUDA path through the C interface against the CPU oracle.

Bar (FP64 mode): max relative error <= 1e-10 on rho, u, T (field-normwise:
max|gpu - oracle| / max|oracle|, u as a vector) after the stated steps; the
two sides differ only in summation order and in the division-free limiter
form (Sec. III, reading A6), both Lipschitz, so differences stay at round-off.
Sizes are chosen so the oracle finishes in seconds while the grids span several
32 x 8 tiles with ragged tails.  FP32 deviation mode: L1 relative <= 1e-4 and
max relative <= 1e-3 on rho, u, T; conserved totals drift <= 1e-6 relative.
"""
import math

import numpy as np
import pytest

from _gpu_helpers import fp64_errors, l1_rel, max_rel, run_both, vel_max_rel
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


def _assert_fp64(errs, tol=TOL):
    for k, v in errs.items():
        assert v <= tol, f"{k}: {v:.3e} > {tol:.0e} ({errs})"


def test_sod_1000_steps(orc, lbm):
    p = wl.sod(200, 4)
    s, O = run_both(orc, lbm, p, 1000)
    _assert_fp64(fp64_errors(s, O))


@pytest.mark.parametrize("Pr", [0.5, 1.0, 2.0])
def test_couette_1000_steps(orc, lbm, Pr):
    p = wl.couette(Pr, nx=4, ny=200)
    s, O = run_both(orc, lbm, p, 1000)
    _assert_fp64(fp64_errors(s, O))


def test_shock_interface_reduced(orc, lbm):
    p = wl.shock_interface(nx=150, ny=38, steps=300)      # ragged in both directions
    s, O = run_both(orc, lbm, p, 300)
    _assert_fp64(fp64_errors(s, O))


def test_shear_layer_reduced(orc, lbm):
    p = wl.shear_layer(100, ny=70)                         # same dx, dt as the 100^2 layer
    s, O = run_both(orc, lbm, p, 300)
    _assert_fp64(fp64_errors(s, O))


@pytest.mark.parametrize("limiter", [1, 2])
def test_lax_wendroff_and_upwind_variants(orc, lbm, limiter):
    p = wl.shock_interface(nx=70, ny=20, steps=100)
    s, O = run_both(orc, lbm, p, 100, limiter=limiter)
    _assert_fp64(fp64_errors(s, O))


def test_every_boundary_kind(orc, lbm):
    """NEQ walls on x (moving, heated), fixed equilibrium on y, Pr != 1, ragged grid."""
    p = wl.shear_layer(64, ny=45)
    p.nx, p.ny = 37, 45
    p.rho, p.ux, p.uy, p.T = (np.ascontiguousarray(a[:45, :37]) for a in (p.rho, p.ux, p.uy, p.T))
    p.bc = [(wl.BC_NEQ_WALL, 1.0, 0.0, 0.02, 1.01), (wl.BC_NEQ_WALL, 1.0, 0.0, -0.03, 0.99),
            (wl.BC_EQUILIBRIUM, 1.02, 0.01, 0.0, 1.0), (wl.BC_EQUILIBRIUM, 0.98, -0.01, 0.0, 1.02)]
    s, O = run_both(orc, lbm, p, 200)
    _assert_fp64(fp64_errors(s, O))


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 9), (9, 1), (2, 3), (33, 9), (31, 7)])
def test_degenerate_and_tile_edge_sizes(orc, lbm, nx, ny):
    p = wl.shear_layer(64, ny=max(ny, 1))
    p.nx, p.ny = nx, ny
    rng = np.random.default_rng(nx * 100 + ny)
    p.rho = 1.0 + 0.05 * rng.uniform(-1, 1, (ny, nx))
    p.ux = 0.05 * rng.uniform(-1, 1, (ny, nx))
    p.uy = 0.05 * rng.uniform(-1, 1, (ny, nx))
    p.T = 1.0 + 0.05 * rng.uniform(-1, 1, (ny, nx))
    s, O = run_both(orc, lbm, p, 50)
    _assert_fp64(fp64_errors(s, O))


def test_delta_and_delta_star(orc, lbm):
    p = wl.shock_interface(nx=96, ny=24, steps=150)
    s, O = run_both(orc, lbm, p, 150)
    g = s.moments(delta=True)[4]
    r = O.moments(delta=True)[4]
    sc = np.abs(r[4:]).max()
    assert np.abs(g - r).max() <= 1e-9 * sc
    gs = s.moments_central()
    rs = O.moments_central()
    assert np.abs(gs - rs).max() <= 1e-9 * np.abs(rs[4:]).max()


def test_totals_and_state_roundtrip(orc, lbm):
    p = wl.shear_layer(64, ny=40)
    s, O = run_both(orc, lbm, p, 100)
    tg, to = s.totals(), O.totals()
    assert np.abs(tg - to).max() <= 1e-12 * np.abs(to).max()
    fg, fo = s.get_state(), O.get_state()
    assert np.abs(fg - fo).max() <= 1e-10 * np.abs(fo).max()
    rows = s.get_state_rows(10, 7)
    assert np.array_equal(rows, fg[:, 10:17, :])
    s.set_state(fo)                                    # continue both from the oracle's state
    s.step(20)
    O.step(20)
    _assert_fp64(fp64_errors(s, O))
    assert s.step_count == 20


def test_periodic_totals_conserved_on_gpu(lbm):
    p = wl.shear_layer(128)
    s = lbm.Solver.from_problem(p)
    s.init(*p.fields())
    t0 = s.totals()
    s.step(500)
    t1 = s.totals()
    assert np.abs(t1 - t0).max() <= 1e-12 * np.abs(t0).max()


def test_step_before_init_and_bad_n(lbm):
    p = wl.sod(200, 2)
    s = lbm.Solver.from_problem(p)
    with pytest.raises(lbm.LbmError) as e:
        s.step(1)
    assert e.value.code == lbm.LBM_ERR_STATE
    s.init(*p.fields())
    with pytest.raises(lbm.LbmError) as e:
        s.step(0)
    assert e.value.code == lbm.LBM_ERR_STATE


@pytest.mark.parametrize("field,value", [(0, 0.0), (0, -1.0), (1, float("nan")), (3, 0.0), (2, float("inf"))])
def test_invalid_init_fields_are_rejected_on_the_device(lbm, field, value):
    """lbm_init checks rho > 0, T > 0 and finiteness in the init kernel: one bad cell (in the
    second of several staging chunks) gives LBM_ERR_ARG and leaves the context uninitialised;
    a valid init afterwards works."""
    p = wl.shear_layer(1600, ny=1500)                    # 2.4 M cells: two staging chunks
    bad = [np.array(a, copy=True) for a in p.fields()]
    bad[field][1400, 777] = value
    s = lbm.Solver.from_problem(p, precision=1)
    with pytest.raises(lbm.LbmError) as e:
        s.init(*bad)
    assert e.value.code == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LbmError) as e:
        s.step(1)
    assert e.value.code == lbm.LBM_ERR_STATE
    s.init(*p.fields())
    s.step(2)
    assert np.isfinite(s.moments()[0]).all()
    s.close()


def test_nonfinite_state_is_reported(lbm):
    p = wl.sod(200, 2)
    s = lbm.Solver.from_problem(p)
    s.init(*p.fields())
    f = s.get_state()
    f[3, 1, 57] = np.nan
    s.set_state(f)
    with pytest.raises(lbm.LbmError) as e:
        s.moments()
    assert e.value.code == lbm.LBM_ERR_NONFINITE


# ------------------------------------------------------------------ FP32 deviation mode
def _fp32_errors(s, O):
    g, r = s.moments(), O.moments()
    gu = np.hypot(g[1], g[2])
    du = np.hypot(g[1] - r[1], g[2] - r[2])
    ou = np.hypot(r[1], r[2])
    return {
        "rho_l1": l1_rel(g[0], r[0]), "T_l1": l1_rel(g[3], r[3]), "u_l1": float(du.sum() / ou.sum()),
        "rho_max": max_rel(g[0], r[0]), "T_max": max_rel(g[3], r[3]),
        "u_max": vel_max_rel(g[1], g[2], r[1], r[2]),
    }, gu


@pytest.mark.parametrize("name", ["shear", "sod", "shock"])
def test_fp32_deviation_error_budget(orc, lbm, name):
    if name == "shear":
        p, n = wl.shear_layer(128, ny=96), 400
    elif name == "sod":
        p, n = wl.sod(200, 4), 1000
    else:
        p, n = wl.shock_interface(nx=128, ny=32, steps=300), 300
    s, O = run_both(orc, lbm, p, n, precision=lbm.LBM_FP32_DEV)
    e, _ = _fp32_errors(s, O)
    for k in ("rho_l1", "T_l1", "u_l1"):
        assert e[k] <= 1e-4, e
    for k in ("rho_max", "T_max", "u_max"):
        assert e[k] <= 1e-3, e


def test_fp32_totals_drift(lbm):
    p = wl.shear_layer(256)
    s = lbm.Solver.from_problem(p, precision=lbm.LBM_FP32_DEV)
    s.init(*p.fields())
    t0 = s.totals()
    s.step(500)
    t1 = s.totals()
    for k in (0, 3):                                   # mass and energy (momentum totals are ~0)
        assert abs(t1[k] - t0[k]) <= 1e-6 * abs(t0[k])
    assert np.abs(t1[1:3] - t0[1:3]).max() <= 1e-6 * abs(t0[0])


def test_shock_interface_full_size_100_steps(orc, lbm):
    """The 4096 x 1024 shock-interface problem in full (every cell): 100 steps on the GPU
    against the oracle, float64 to 1e-10 and the float32 deviation mode within its budget."""
    p = wl.shock_interface()
    O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, p.limiter, p.bc)
    O.init(*p.fields())
    O.step(100)
    for prec in (0, 1):
        s = lbm.Solver.from_problem(p, precision=prec)
        s.init(*p.fields())
        s.step(100)
        if prec == 0:
            _assert_fp64(fp64_errors(s, O))
        else:
            e, _ = _fp32_errors(s, O)
            for k in ("rho_l1", "T_l1", "u_l1"):
                assert e[k] <= 1e-4, e
            for k in ("rho_max", "T_max", "u_max"):
                assert e[k] <= 1e-3, e
        s.close()


# ------------------------------------------------------------------ full size, sampled
def _patch(f_rows, y_local, x, nx):
    """[16][5][5] neighbourhood (periodic in x) of cell (x, y_local) from a row window."""
    out = np.zeros((16, 5, 5))
    for dy in range(-2, 3):
        for dx in range(-2, 3):
            if dx != 0 and dy != 0:
                continue
            out[:, dy + 2, dx + 2] = f_rows[:, y_local + dy, (x + dx) % nx]
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_shear_layer_sampled(orc, lbm, prec):
    """8192 x 8192 shear layer (float64: the streaming kernel, the float64-pipe kernel of large
    grids; the automatic double-float kernel has the same check in test_gpu_dd.py; float32
    deviation mode: the TMA-staged tile kernel of the benchmark's launch configuration): after 3
    steps, 64 seeded cells of step 4 are recomputed by the oracle from the GPU's step-3 state.
    float64: 1e-13 of f.
    float32: 1e-6 of f, and per cell 2^-20 (8 float32 ulps) of the cell's largest stored
    deviation |g| = |f - f^eq0| (measured: under 2 ulps).  That is about 1% of the largest
    change of f in the step here, so a dropped or wrong term of the update fails."""
    p = wl.shear_layer(8192)
    s = lbm.Solver.from_problem(p, precision=prec, step_kernel=5 if prec == 0 else 0)
    assert s.step_kernel == (5 if prec == 0 else 2)
    s.init(*p.fields())
    s.step(3)
    rng = np.random.default_rng(7)
    ys = rng.integers(2, p.ny - 2, 64)
    xs = rng.integers(0, p.nx, 64)
    before = {int(y): s.get_state_rows(int(y) - 2, 5) for y in set(ys.tolist())}
    s.step(1)
    O = orc.Oracle(4, 4, p.dx, p.dt, p.gamma, p.s, p.limiter, wl.periodic_bc())
    O.init(np.ones((4, 4)), np.zeros((4, 4)), np.zeros((4, 4)), np.ones((4, 4)))
    feq0 = O.get_state()[:, 0, 0]                      # the float32 mode's reference (1, 0, 0, 1)
    worst, worst_g, largest_change = 0.0, 0.0, 0.0
    for y, x in zip(ys.tolist(), xs.tolist()):
        want = orc.update_patch(_patch(before[y], 2, x, p.nx), p.dx, p.dt, p.gamma, p.s, p.limiter)
        got = s.get_state_rows(y, 1)[:, 0, x]
        prev = before[y][:, 2, x]
        worst = max(worst, np.abs(got - want).max() / np.abs(want).max())
        worst_g = max(worst_g, np.abs(got - want).max() / np.abs(prev - feq0).max())
        largest_change = max(largest_change, np.abs(want - prev).max())
    s.close()
    if prec == 0:
        assert worst <= 1e-13
    else:
        assert worst <= 1e-6
        assert worst_g <= 2.0 ** -20, (worst_g, largest_change)


# ------------------------------------------------------------------ TMA-staged kernel == plain kernel
def _state_after(lbm, p, steps, precision, kernel, limiter=None):
    s = lbm.Solver(p.nx, p.ny, p.dx, p.dt, p.gamma, p.Pr, p.s, p.limiter if limiter is None else limiter,
                   p.bc, precision=precision, step_kernel=kernel)
    s.init(*p.fields())
    s.step(steps)
    out = s.get_state()
    s.close()
    return out


# The two kernels do the same arithmetic per value; only the compiler's multiply-add
# contraction may differ, so they agree to round-off of the storage precision.
ROUNDOFF = {0: 1e-13, 1: 2e-5}


def _assert_roundoff(a, b, precision):
    assert np.abs(a - b).max() <= ROUNDOFF[precision] * np.abs(b).max()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("limiter", [0, 1, 2])
def test_tma_kernel_matches_plain_kernel(lbm, precision, limiter):
    p = wl.shock_interface(nx=150, ny=70, steps=60)          # ragged against 32 x 32 tiles
    a = _state_after(lbm, p, 60, precision, 1, limiter)
    b = _state_after(lbm, p, 60, precision, 2, limiter)
    _assert_roundoff(a, b, precision)


@pytest.mark.parametrize("limiter", [0, 1, 2])
def test_tma_kernel_each_limiter_against_oracle(orc, lbm, limiter):
    p = wl.shock_interface(nx=150, ny=70, steps=120)
    s = lbm.Solver(p.nx, p.ny, p.dx, p.dt, p.gamma, p.Pr, p.s, limiter, p.bc, step_kernel=2)
    s.init(*p.fields())
    s.step(120)
    O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, limiter, p.bc)
    O.init(*p.fields())
    O.step(120)
    _assert_fp64(fp64_errors(s, O))
    fo = O.get_state()
    assert np.abs(s.get_state() - fo).max() <= TOL * np.abs(fo).max()


def test_fp32_state_roundtrip_against_oracle(orc, lbm):
    """get_state / set_state in the deviation mode return and accept f (not g)."""
    p = wl.shock_interface(nx=96, ny=40, steps=50)
    s, O = run_both(orc, lbm, p, 50, precision=lbm.LBM_FP32_DEV)
    fg, fo = s.get_state(), O.get_state()
    assert np.abs(fg - fo).max() <= 1e-4 * np.abs(fo).max()
    s.set_state(fo)
    assert np.abs(s.get_state() - fo).max() <= 1e-6 * np.abs(fo).max()   # float32 storage of g


@pytest.mark.parametrize("precision", [0, 1])
def test_tma_kernel_matches_plain_kernel_walls(lbm, precision):
    p = wl.shear_layer(64, ny=45)
    p.nx, p.ny = 61, 45
    p.rho, p.ux, p.uy, p.T = (np.ascontiguousarray(a[:45, :61]) for a in (p.rho, p.ux, p.uy, p.T))
    p.bc = [(wl.BC_NEQ_WALL, 1.0, 0.0, 0.02, 1.01), (wl.BC_NEQ_WALL, 1.0, 0.0, -0.03, 0.99),
            (wl.BC_EQUILIBRIUM, 1.02, 0.01, 0.0, 1.0), (wl.BC_ZERO_GRADIENT, 0, 0, 0, 0)]
    p.bc[3] = (wl.BC_ZERO_GRADIENT, 0, 0, 0, 0)
    p.bc[2] = (wl.BC_ZERO_GRADIENT, 0, 0, 0, 0)
    a = _state_after(lbm, p, 80, precision, 1)
    b = _state_after(lbm, p, 80, precision, 2)
    _assert_roundoff(a, b, precision)


def test_tma_kernel_parity_with_oracle(orc, lbm):
    p = wl.shear_layer(96, ny=66)
    p.bc = [(wl.BC_NEQ_WALL, 1.0, 0.0, 0.02, 1.01), (wl.BC_NEQ_WALL, 1.0, 0.0, -0.03, 0.99),
            (wl.BC_PERIODIC, 0, 0, 0, 0), (wl.BC_PERIODIC, 0, 0, 0, 0)]
    s = lbm.Solver(p.nx, p.ny, p.dx, p.dt, p.gamma, p.Pr, p.s, p.limiter, p.bc, step_kernel=2)
    s.init(*p.fields())
    s.step(300)
    O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, p.limiter, p.bc)
    O.init(*p.fields())
    O.step(300)
    _assert_fp64(fp64_errors(s, O))


# ------------------------------------------------------------------ 1000 steps, reduced C3 / C4
@pytest.mark.parametrize("name", ["shock_interface_512x128", "shear_layer_1024x1024"])
def test_reduced_configs_1000_steps_every_fp64_kernel(orc, lbm, name):
    """The shock-interface and shear-layer configurations reduced to 512 x 128 and 1024 x 1024
    (same physics), 1000 steps: the automatic float64 kernel, the streaming kernel and the
    TMA-staged tile kernel each match one oracle run to 1e-10 on rho, u, T."""
    p = (wl.shock_interface(nx=512, ny=128, steps=1000) if name.startswith("shock")
         else wl.shear_layer(1024, steps=1000))
    O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, p.limiter, p.bc)
    O.init(*p.fields())
    O.step(1000)
    for kernel in (0, 5, 2):
        s = lbm.Solver.from_problem(p, step_kernel=kernel)
        s.init(*p.fields())
        s.step(1000)
        errs = fp64_errors(s, O)
        s.close()
        for k, v in errs.items():
            assert v <= TOL, f"kernel {kernel}, {k}: {v:.3e} ({errs})"
