"""The C interface without a GPU: the library loads, exports every function
include/lbm.h declares, and rejects invalid arguments on the host before any
device work (status codes of include/lbm.h)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1305_4736_gb300 import build, lbm
    build.build()
    return lbm


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 13
    L = lib.load()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(lib.EXPORTS)


def _good():
    from paper_1305_4736_gb300 import workloads as wl
    p = wl.sod(200, 4)
    return dict(nx=p.nx, ny=p.ny, dx=p.dx, dt=p.dt, gamma=p.gamma, Pr=1.0, s=p.s.copy(),
                limiter=0, bc=p.bc)


def _create_rc(lib, **kw):
    a = _good()
    a.update(kw)
    L = lib.load()
    h = ctypes.c_void_p()
    s = np.ascontiguousarray(a["s"], dtype=np.float64)
    bc = lib.make_bc(a["bc"])
    rc = L.lbm_create(a["nx"], a["ny"], a["dx"], a["dt"], a["gamma"], a["Pr"], s.ctypes.data_as(lib._D),
                      a["limiter"], ctypes.byref(bc), ctypes.byref(h))
    if rc == 0:
        L.lbm_destroy(h)
    return rc, L.lbm_last_error(None).decode()


@pytest.mark.parametrize("kw,code", [
    (dict(nx=0), -1), (dict(ny=-3), -1), (dict(dx=0.0), -1), (dict(dt=-1e-4), -1),
    (dict(gamma=1.0), -1), (dict(Pr=0.0), -1), (dict(limiter=7), -1),
    (dict(dt=1e-3, s=np.full(16, 100.0)), -2),             # 6 dt/dx = 1.2 > 1
    (dict(s=np.full(16, 3e4)), -3),                        # s dt = 3 >= 2
    (dict(nx=1 << 16, ny=1 << 15), -1),                     # 2^31 cells: above the grid limit
    (dict(nx=(1 << 28) + 1, ny=1), -1),                     # a side above 2^28
])
def test_create_rejects_bad_arguments(lib, kw, code):
    rc, msg = _create_rc(lib, **kw)
    assert rc == code and msg


def test_isotropy_and_prandtl_checks(lib):
    s = np.full(16, 1e3)
    s[5] = 2e3                                             # s6 != s5
    assert _create_rc(lib, s=s)[0] == -1
    s = np.full(16, 1e3)
    s[7] = s[8] = 500.0
    assert _create_rc(lib, s=s, Pr=1.0)[0] == -1          # Pr != s8/s5
    s2 = s.copy()
    s2[8] = 600.0
    assert _create_rc(lib, s=s2, Pr=0.5)[0] == -1         # s8 != s9


def test_periodic_pairing_and_edge_states(lib):
    bc = [(1, 0, 0, 0, 0), (0, 0, 0, 0, 0), (0, 0, 0, 0, 0), (0, 0, 0, 0, 0)]
    assert _create_rc(lib, bc=bc)[0] == -1
    bc = [(2, -1.0, 0, 0, 1.0), (2, 1.0, 0, 0, 1.0), (0, 0, 0, 0, 0), (0, 0, 0, 0, 0)]
    assert _create_rc(lib, bc=bc)[0] == -1                # equilibrium rho <= 0
    bc = [(3, 1.0, 0, 0, 0.0), (3, 1.0, 0, 0, 1.0), (0, 0, 0, 0, 0), (0, 0, 0, 0, 0)]
    assert _create_rc(lib, bc=bc)[0] == -1                # wall T <= 0
    bc = [(9, 1.0, 0, 0, 1.0), (1, 1.0, 0, 0, 1.0), (0, 0, 0, 0, 0), (0, 0, 0, 0, 0)]
    assert _create_rc(lib, bc=bc)[0] == -1                # unknown kind


def test_null_safety_and_footprint(lib):
    L = lib.load()
    L.lbm_destroy(None)
    assert L.lbm_step(None, 1) == -1
    assert L.lbm_totals(None, None) == -1
    assert L.lbm_step_count(None) == -1
    assert lib.lbm_footprint(200, 4, 0) == 2 * 16 * 8 * 224 * 8
    assert lib.lbm_footprint(200, 4, 1) == 2 * 16 * 8 * 224 * 4
    assert lib.lbm_footprint(0, 4, 0) == 0
    assert lib.lbm_footprint(8192, 8192, 0) == 2 * 16 * 8196 * 8224 * 8


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="checks the no-GPU path")
def test_valid_create_without_gpu_reports_cuda_error(lib):
    rc, msg = _create_rc(lib)
    assert rc in (-5, -4) and msg
