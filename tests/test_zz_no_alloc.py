"""lbm_totals_noalloc: conserved totals computed with no device allocation.

It serves callers that cannot allocate device memory (their memory belongs to
another allocator, or they must not call cudaMalloc / cudaFree, which can
synchronise the device).  The test hands it a population field that the test
itself placed on the GPU and checks, on two calls in a row, that it returns the
totals lbm_totals gives for the same state.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1305_4736_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_totals_noalloc_matches_lbm_totals_on_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1305_4736_gb300 import build, lbm
    build.build()
    L = lbm.load()
    p = wl.shear_layer(128, ny=96)
    s = lbm.Solver.from_problem(p)
    s.init(*p.fields())
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        if call == 1:
            s.step(50)                                    # a different state for the second call
        ref = s.totals()
        f = torch.from_numpy(s.get_state()).cuda()        # [16][ny][nx] float64 on the device
        torch.cuda.synchronize()
        out = np.zeros(4)
        rc = L.lbm_totals_noalloc(ctypes.c_void_p(f.data_ptr()), p.nx, p.ny, p.dx, ctypes.c_void_p(stream),
                                  out.ctypes.data_as(lbm._D))
        assert rc == lbm.LBM_OK
        assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()
    too_many = lbm.LBM_OK
    out = np.zeros(4)
    too_many = L.lbm_totals_noalloc(ctypes.c_void_p(f.data_ptr()), 1, 16385, p.dx, ctypes.c_void_p(stream),
                                    out.ctypes.data_as(lbm._D))
    assert too_many == lbm.LBM_ERR_ARG
    s.close()
