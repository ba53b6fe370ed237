"""lbm_step's graph replay (runs of 16 steps or more as pairs of steps from a per-context CUDA
graph) against stepping one step per call (direct launches): bit-identical on every kernel
family, for odd run lengths and either starting buffer, and after lbm_autotune has changed the
kernel (which drops the captured graphs)."""
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


CASES = [
    ("sod_fp64_narrow", lambda: wl.sod(200, 4), 0, 0, 9),
    ("sod_fp32_plain", lambda: wl.sod(200, 4), 1, 0, 1),
    ("shear_fp64_wide", lambda: wl.shear_layer(512, ny=320), 0, 0, 8),
    ("shear_fp32_tile", lambda: wl.shear_layer(256, ny=128), 1, 0, 2),
    ("couette_fp64_plain", lambda: wl.couette(2.0, nx=4, ny=200), 0, 0, 7),
    ("shear_fp64_stream", lambda: wl.shear_layer(256, ny=64), 0, 5, 5),
]


def _make(lbm, mk, prec, kernel):
    p = mk()
    s = lbm.Solver.from_problem(p, precision=prec, step_kernel=kernel)
    s.init(*p.fields())
    return s


@pytest.mark.parametrize("name,mk,prec,kernel,want", CASES, ids=[c[0] for c in CASES])
def test_graph_runs_equal_single_steps(lbm, name, mk, prec, kernel, want):
    a, b = _make(lbm, mk, prec, kernel), _make(lbm, mk, prec, kernel)
    assert a.step_kernel == want and b.step_kernel == want
    # a: one direct step (odd parity), then runs of 33 and 40 steps (graph pairs from either
    # starting buffer plus a direct step); b: the same 74 steps one per call
    a.step(1)
    a.step(33)
    a.step(40)
    for _ in range(74):
        b.step(1)
    assert a.step_count == b.step_count == 74
    assert np.array_equal(a.get_state(), b.get_state())
    a.close()
    b.close()


def test_graph_after_autotune(lbm):
    """lbm_autotune drops the captured graphs: the next run replays the chosen kernel, bit for
    bit as a context created on that kernel and stepped one step per call."""
    p = wl.shear_layer(512, ny=320)
    a = lbm.Solver.from_problem(p)
    a.init(*p.fields())
    a.step(20)                                  # captures the pair graph of the automatic kernel
    choice = a.autotune(2)
    state = a.get_state()
    b = lbm.Solver.from_problem(p, step_kernel=choice)
    b.set_state(state)
    a.step(32)
    for _ in range(32):
        b.step(1)
    assert np.array_equal(a.get_state(), b.get_state())
    a.close()
    b.close()
