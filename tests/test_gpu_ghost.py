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
