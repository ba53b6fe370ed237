"""GPU parity of the ghost fill on the x edges (Sec. IV: periodic and zero-gradient edges).

With an even nx, the periodic and zero-gradient x edges copy both ghost columns of a row
in one 16-byte access per population (pair) plane. An odd nx takes the per-cell copy.
Both forms are compared with the oracle after 40 steps: float64 at the 1e-10 bar and
float32 deviation storage within its round-off budget. The cases cover both kinds (a
periodic edge is always paired), even and odd widths, and widths of 2 and 3 cells.
"""
import numpy as np
import pytest

from _gpu_helpers import fp64_errors, l1_rel, max_rel, run_both
from paper_1305_4736_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-10
P = (wl.BC_PERIODIC, 0.0, 0.0, 0.0, 0.0)
Z = (wl.BC_ZERO_GRADIENT, 0.0, 0.0, 0.0, 0.0)


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1305_4736_gb300 import build, lbm as L
    build.build()
    L.load()
    return L


def _problem(nx, ny, xlo, xhi):
    p = wl.shear_layer(max(nx, ny, 16), seed=12, steps=40)
    p.nx, p.ny = nx, ny
    p.rho, p.ux, p.uy, p.T = (np.ascontiguousarray(a[:ny, :nx]) for a in (p.rho, p.ux, p.uy, p.T))
    # a uniform inflow jet along x on top of the layer, so that the x edges carry flux
    p.ux = p.ux + 0.02
    p.bc = [xlo, xhi, P, P]
    return p


@pytest.mark.parametrize("nx", [64, 65, 2, 3])
@pytest.mark.parametrize("edges", [(P, P), (Z, Z)], ids=["per-per", "zg-zg"])
def test_fp64_x_ghost_against_oracle(orc, lbm, nx, edges):
    p = _problem(nx, 24, *edges)
    s, O = run_both(orc, lbm, p, 40)
    errs = fp64_errors(s, O)
    fo = O.get_state()
    got = s.get_state()
    s.close()
    for k, v in errs.items():
        assert v <= TOL, f"{k}: {v:.3e} ({errs})"
    assert np.abs(got - fo).max() <= TOL * np.abs(fo).max()


@pytest.mark.parametrize("nx", [96, 97])
@pytest.mark.parametrize("edges", [(P, P), (Z, Z)], ids=["per-per", "zg-zg"])
def test_fp32_x_ghost_against_oracle(orc, lbm, nx, edges):
    p = _problem(nx, 40, *edges)
    s, O = run_both(orc, lbm, p, 40, precision=lbm.LBM_FP32_DEV)
    g, r = s.moments(), O.moments()
    s.close()
    for a, b in ((g[0], r[0]), (g[3], r[3])):
        assert l1_rel(a, b) <= 1e-4 and max_rel(a, b) <= 1e-3


# ---- the TMA-staged tile kernel without ghost fill on periodic grids
def _periodic(nx, ny, seed=14):
    p = wl.shear_layer(max(nx, ny), seed=seed, steps=40)
    p.nx, p.ny = nx, ny
    p.rho, p.ux, p.uy, p.T = (np.ascontiguousarray(a[:ny, :nx]) for a in (p.rho, p.ux, p.uy, p.T))
    p.ux = p.ux + 0.02
    return p


def _tma(lbm, p, precision, kernel=2):
    s = lbm.Solver(p.nx, p.ny, p.dx, p.dt, p.gamma, p.Pr, p.s, p.limiter, p.bc, precision=precision,
                   step_kernel=kernel)
    s.init(*p.fields())
    return s


@pytest.mark.parametrize("nx,ny", [(32, 32), (33, 35), (70, 50)])
def test_fp64_tile_kernel_wraps_periodic_edges(orc, lbm, nx, ny):
    """Tiles at a periodic edge take their halo from the wrapped interior (no ghost fill on a
    doubly periodic grid); the smallest grid of one tile and ragged grids, against the oracle."""
    p = _periodic(nx, ny)
    s = _tma(lbm, p, 0)
    s.step(40)
    O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, p.limiter, p.bc)
    O.init(*p.fields())
    O.step(40)
    fo = O.get_state()
    got = s.get_state()
    s.close()
    assert np.abs(got - fo).max() <= TOL * np.abs(fo).max()


@pytest.mark.parametrize("nx,ny", [(32, 16), (33, 17), (45, 30), (96, 64)])
def test_fp32_tile_kernel_wraps_periodic_edges(lbm, nx, ny):
    p = _periodic(nx, ny)
    a, b = _tma(lbm, p, 1, kernel=1), _tma(lbm, p, 1, kernel=2)
    a.step(40)
    b.step(40)
    want, got = a.get_state(), b.get_state()
    a.close()
    b.close()
    assert np.abs(got - want).max() <= 2e-5 * np.abs(want).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_tile_kernel_periodic_in_x_walls_in_y(orc, lbm, precision):
    """One periodic axis: the x halo wraps in the kernel, the y walls come from the ghost fill."""
    p = _periodic(64, 40)
    p.bc = [P, P, (wl.BC_NEQ_WALL, 1.0, 0.01, 0.0, 1.0), (wl.BC_NEQ_WALL, 1.0, -0.02, 0.0, 1.01)]
    s = _tma(lbm, p, precision)
    s.step(40)
    O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, p.limiter, p.bc)
    O.init(*p.fields())
    O.step(40)
    if precision == 0:
        fo = O.get_state()
        assert np.abs(s.get_state() - fo).max() <= TOL * np.abs(fo).max()
    else:
        g, r = s.moments(), O.moments()
        for a, b in ((g[0], r[0]), (g[3], r[3])):
            assert l1_rel(a, b) <= 1e-4 and max_rel(a, b) <= 1e-3
    s.close()
