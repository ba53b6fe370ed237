"""Host transfers of lbm_init and lbm_moments.

Page-locked host arrays (a pinned torch tensor) are read and written by the init and
moments kernels over the host link; other host memory goes through the chunked staging
buffer. The two routes run the same per-cell arithmetic, so their results are identical
bit for bit. That holds for ρ, u, v, T, Δ and Δ*, for both precisions, and for a grid
larger than one staging chunk. The float32 deviation mode evaluates its initial deviation
g = f^eq - f^eq0 in float32 from float64 deviations of ρ, j and P. Its initial state is
pinned against the oracle's f^eq at a few float32 roundings of g.
"""
import numpy as np
import pytest

from paper_1305_4736_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1305_4736_gb300 import build, lbm as L
    build.build()
    L.load()
    return L


def _pinned(shape, fill=None):
    import torch
    t = torch.empty(shape, dtype=torch.float64, pin_memory=True)
    a = t.numpy()
    if fill is not None:
        np.copyto(a, fill)
    return a, t


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n", [96, 1600])          # 1600^2: several staging chunks
def test_pinned_and_pageable_paths_agree(lbm, precision, n):
    p = wl.shear_layer(n, seed=21)
    pinned = [_pinned(a.shape, a) for a in p.fields()]
    a = lbm.Solver.from_problem(p, precision=precision)
    a.init(*(x for x, _ in pinned))
    b = lbm.Solver.from_problem(p, precision=precision)
    b.init(*(np.array(x) for x in p.fields()))
    assert np.array_equal(a.get_state(), b.get_state())
    a.step(5)
    b.step(5)
    outs = [_pinned((p.ny, p.nx)) for _ in range(4)]
    dl = _pinned((16, p.ny, p.nx)) if n <= 96 else (None, None)
    rc = lbm.lbm_moments(a.h, outs[0][0], outs[1][0], outs[2][0], outs[3][0], dl[0])
    assert rc == lbm.LBM_OK
    want = b.moments(delta=n <= 96)
    for got, w in zip([o for o, _ in outs] + ([dl[0]] if n <= 96 else []), want):
        assert np.array_equal(got, w)
    if n <= 96:
        ds = _pinned((16, p.ny, p.nx))
        lbm.lbm_moments_central(a.h, ds[0])
        assert np.array_equal(ds[0], b.moments_central())
    a.close()
    b.close()


def test_pinned_init_rejects_a_bad_cell(lbm):
    p = wl.shear_layer(256)
    fields = [_pinned(a.shape, a) for a in p.fields()]
    fields[3][0][200, 17] = -1.0
    s = lbm.Solver.from_problem(p, precision=1)
    with pytest.raises(lbm.LbmError) as e:
        s.init(*(x for x, _ in fields))
    assert e.value.code == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LbmError):
        s.step(1)
    s.close()


def test_moments_mixing_pinned_and_pageable_outputs(lbm):
    """One pageable output sends every output through the staging buffer."""
    p = wl.shear_layer(128, seed=4)
    s = lbm.Solver.from_problem(p)
    s.init(*p.fields())
    s.step(3)
    rho_p = _pinned((p.ny, p.nx))
    u = np.empty((p.ny, p.nx))
    rc = lbm.lbm_moments(s.h, rho_p[0], u, None, None, None)
    assert rc == lbm.LBM_OK
    want = s.moments()
    assert np.array_equal(rho_p[0], want[0]) and np.array_equal(u, want[1])
    s.close()


@pytest.mark.parametrize("name", ["shear", "shock"])
def test_fp32_initial_state_against_oracle(orc, lbm, name):
    p = wl.shear_layer(128, ny=64) if name == "shear" else wl.shock_interface(nx=128, ny=32, steps=1)
    s = lbm.Solver.from_problem(p, precision=lbm.LBM_FP32_DEV)
    s.init(*p.fields())
    got = s.get_state()
    s.close()
    O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, p.limiter, p.bc)
    O.init(*p.fields())
    fo = O.get_state()
    # |g| = |f - f^eq0| is of the order of the spread of each population over the domain;
    # float32 evaluation and storage of g stay within 1e-6 of that spread
    spread = np.abs(fo - fo.mean(axis=(1, 2), keepdims=True)).max()
    assert np.abs(got - fo).max() <= 1e-6 * max(spread, 1e-3)


@pytest.mark.parametrize("precision", [0, 1])
def test_state_round_trip_through_pinned_memory(lbm, precision):
    """lbm_get_state, lbm_get_state_rows and lbm_set_state on page-locked arrays give the
    staged route's results bit for bit."""
    p = wl.shear_layer(700, ny=1300, seed=7)          # 0.9 M cells: two staging chunks of 16 planes
    s = lbm.Solver.from_problem(p, precision=precision)
    s.init(*p.fields())
    s.step(3)
    want = s.get_state()
    got, _t = _pinned(want.shape)
    lbm.lbm_get_state(s.h, got)
    assert np.array_equal(got, want)
    rows, _r = _pinned((16, 301, p.nx))
    lbm.lbm_get_state_rows(s.h, 555, 301, rows)
    assert np.array_equal(rows, want[:, 555:856])
    # write back a perturbed state through the pinned route, read it through the staged route
    new, _n = _pinned(want.shape, want * (1.0 + 1e-3))
    lbm.lbm_set_state(s.h, new)
    back = s.get_state()
    t = lbm.Solver.from_problem(p, precision=precision)
    t.set_state(np.array(new))
    assert np.array_equal(back, t.get_state())
    s.close()
    t.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_and_resume_in_a_new_context(lbm, precision):
    """30 steps, lbm_get_state into a page-locked checkpoint, a new context resumed from it with
    lbm_set_state, 30 more steps: the same state as 60 uninterrupted steps.  float64: bit for
    bit.  float32: g goes through f = g + f^eq0 in float64 and back, so the resumed state may
    differ in the last bit of g; bounded by the storage precision."""
    p = wl.shear_layer(384, ny=200, seed=31)
    ref = lbm.Solver.from_problem(p, precision=precision)
    ref.init(*p.fields())
    ref.step(60)
    want = ref.get_state()
    ref.close()
    a = lbm.Solver.from_problem(p, precision=precision)
    a.init(*p.fields())
    a.step(30)
    ckpt, _t = _pinned((16, p.ny, p.nx))
    lbm.lbm_get_state(a.h, ckpt)
    a.close()
    b = lbm.Solver.from_problem(p, precision=precision)
    lbm.lbm_set_state(b.h, ckpt)
    b.step(30)
    got = b.get_state()
    b.close()
    if precision == 0:
        assert np.array_equal(got, want)
    else:
        assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max()
