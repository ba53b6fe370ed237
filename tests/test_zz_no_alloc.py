"""lbm_totals_noalloc: conserved totals computed with no device allocation.

It serves callers that cannot allocate device memory (their memory belongs to
another allocator, or they must not call cudaMalloc / cudaFree, which can
synchronise the device).  The test hands it a population field that the test
itself placed on the GPU and checks, on two calls in a row, that it returns the
totals lbm_totals gives for the same state and the totals the oracle computes
from the same populations, on a grid with dy = dx and on one with dy != dx (the
totals are sums times the cell area dx dy).  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1305_4736_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dy_ratio", [1.0, 0.6])
def test_totals_noalloc_matches_lbm_totals_and_oracle_on_two_calls(orc, dy_ratio):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1305_4736_gb300 import build, lbm
    build.build()
    L = lbm.load()
    p = wl.shear_layer(128, ny=96)
    p.dy = dy_ratio * p.dx
    s = lbm.Solver.from_problem(p)
    s.init(*p.fields())
    O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, p.limiter, p.bc, dy=p.dy)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        if call == 1:
            s.step(50)                                    # a different state for the second call
        ref = s.totals()
        state = s.get_state()
        O.set_state(state)
        ref_oracle = O.totals()
        f = torch.from_numpy(state).cuda()                # [16][ny][nx] float64 on the device
        torch.cuda.synchronize()
        out = np.zeros(4)
        rc = L.lbm_totals_noalloc(ctypes.c_void_p(f.data_ptr()), p.nx, p.ny, p.dx, p.dy,
                                  ctypes.c_void_p(stream), out.ctypes.data_as(lbm._D))
        assert rc == lbm.LBM_OK
        assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()
        assert np.abs(out - ref_oracle).max() <= 1e-12 * np.abs(ref_oracle).max()
    out = np.zeros(4)
    too_many = L.lbm_totals_noalloc(ctypes.c_void_p(f.data_ptr()), 1, 16385, p.dx, p.dy,
                                    ctypes.c_void_p(stream), out.ctypes.data_as(lbm._D))
    assert too_many == lbm.LBM_ERR_ARG
    bad_dy = L.lbm_totals_noalloc(ctypes.c_void_p(f.data_ptr()), p.nx, p.ny, p.dx, 0.0,
                                  ctypes.c_void_p(stream), out.ctypes.data_as(lbm._D))
    assert bad_dy == lbm.LBM_ERR_ARG
    s.close()
    O.close()
