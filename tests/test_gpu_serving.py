"""Serving loop on the GPU: every request's result is the same alone and in the mix
(bit for bit: the batched kernel's tiles are independent), the mix really overlaps
requests on the device, and float64 results match the oracle (<= 1e-10)."""
import numpy as np
import pytest

from _gpu_helpers import max_rel, vel_max_rel
from paper_1305_4736_gb300 import serving, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def backend():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1305_4736_gb300 import build
    build.build()
    return serving.GpuBackend()


def test_results_same_alone_and_in_mix(orc, backend):
    reqs = wl.serving_requests(count=9, seed=11, rate_hz=1000.0, max_nx=200, max_ny=40, steps=150)
    mix, st = serving.Engine(backend, chunk=40, realtime=False).run(reqs)
    assert st.solves == len(reqs) and st.max_resident_solves >= 3
    for r in reqs:
        one, _ = serving.Engine(backend, chunk=40, realtime=False).run([dict(r, arrival=0.0)])
        for a, b in zip(one[0].moments, mix[r["id"]].moments):
            assert np.array_equal(a, b), r["id"]
    checked = 0
    for r in reqs:
        if r["precision"] != 0:
            continue
        p = r["problem"]
        O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, p.limiter, p.bc)
        O.init(*p.fields())
        O.step(p.steps)
        o = O.moments()
        g = mix[r["id"]].moments
        assert max_rel(g[0], o[0]) <= 1e-10 and max_rel(g[3], o[3]) <= 1e-10
        assert vel_max_rel(g[1], g[2], o[1], o[2]) <= 1e-10
        checked += 1
    assert checked >= 2
