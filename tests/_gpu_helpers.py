"""Shared helpers of the GPU tests (not collected by pytest)."""
import numpy as np


def run_both(orc, lbm, p, steps, precision=0, limiter=None):
    """Run problem p for `steps` on the GPU (through the C interface) and on the oracle."""
    lim = p.limiter if limiter is None else limiter
    s = lbm.Solver(p.nx, p.ny, p.dx, p.dt, p.gamma, p.Pr, p.s, lim, p.bc, precision=precision, dy=p.dy)
    s.init(*p.fields())
    if steps:
        s.step(steps)
    O = orc.Oracle(p.nx, p.ny, p.dx, p.dt, p.gamma, p.s, lim, p.bc, dy=p.dy)
    O.init(*p.fields())
    if steps:
        O.step(steps)
    return s, O


def max_rel(a, b):
    """max |a - b| / max |b| (field-normwise relative error)."""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def vel_max_rel(gu, gv, ou, ov):
    """max over cells of |u_gpu - u_oracle| (both components) / max |u_oracle|."""
    d = np.maximum(np.abs(gu - ou), np.abs(gv - ov)).max()
    sc = max(np.abs(ou).max(), np.abs(ov).max())
    return float(d / sc) if sc > 1e-12 else float(d)


def l1_rel(a, b):
    return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))


def fp64_errors(s, O):
    g = s.moments()
    r = O.moments()
    return {"rho": max_rel(g[0], r[0]), "u": vel_max_rel(g[1], g[2], r[1], r[2]), "T": max_rel(g[3], r[3])}
