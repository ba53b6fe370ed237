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


# ---- the TMA-staged tile kernel on periodic grids
# On grids of at least 32 waves of tiles (2048 cells per SM a wave; 9.96 M cells on 152 SMs)
# periodic in x, the tile kernel takes the x halo of its edge tiles from the wrapped interior
# and the ghost launch copies only the ghost rows; smaller grids keep the full ghost fill.
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
def test_fp64_tile_kernel_small_periodic_grids(orc, lbm, nx, ny):
    """The tile kernel on periodic grids of one tile and ragged grids, against the oracle."""
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


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("walls_in_y", [False, True])
def test_tile_kernel_wraps_x_halo_on_large_grids(lbm, precision, walls_in_y):
    """3000 x 3500 (10.5 M cells, ragged against the tiles in x and y): the tile kernel with the
    x halo wrapped in the kernel against the plain kernel with the full ghost fill, after 12
    steps (round-off of the storage precision), periodic in y or with walls in y."""
    p = _periodic(3000, 3500, seed=15)
    if walls_in_y:
        p.bc = [P, P, (wl.BC_NEQ_WALL, 1.0, 0.01, 0.0, 1.0), (wl.BC_NEQ_WALL, 1.0, -0.02, 0.0, 1.01)]
    a, b = _tma(lbm, p, precision, kernel=1), _tma(lbm, p, precision, kernel=2)
    a.step(12)
    b.step(12)
    rows = [0, 1, 2, 1747, 3497, 3498, 3499]
    for r0 in rows:
        want, got = a.get_state_rows(r0, 1), b.get_state_rows(r0, 1)
        assert np.isfinite(got).all()
        assert np.abs(got - want).max() <= (1e-13 if precision == 0 else 2e-5) * np.abs(want).max(), r0
    a.close()
    b.close()
