"""Pins against the states the paper prints (tests/golden/paper_printed_states.txt).

- Sec. IV.A: the printed left and right states satisfy the Hugoniot relations for gamma = 2.
  The oracle's exact Riemann solver, given them as Riemann data, returns the left state as the
  star state (to the printed rounding) and a single right-moving shock of speed 2 (no left
  wave of any strength).
- Sec. V: the same shocked state printed in pressure form: p = rho T (R = 1, reading A1) to
  the printed digits, and the incident shock's Mach number 2 / sqrt(gamma p_h / rho_h)
  equals the printed 1.414.
- The workloads transcribe these states: the exact values 3/2, 2/3, 14/9, 7/3 round to the
  printed digits, and the Lax tube uses the printed states as they stand.
"""
import math
import os

import numpy as np
import pytest

from oracle import riemann as R
from paper_1305_4736_gb300 import workloads as wl

HERE = os.path.dirname(__file__)


def _states():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_printed_states.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *pairs = line.split()
            out[key] = {k: float(v) for k, v in (p.split("=") for p in pairs)}
    return out


S = _states()


def _printed_digits_tol(x: float) -> float:
    """Half a unit in the last printed decimal of x (as the fixture writes it)."""
    txt = repr(x)
    dec = len(txt.split(".")[1]) if "." in txt else 0
    return 0.5 * 10.0 ** (-dec) + 1e-12


def test_sec4a_states_are_one_shock_of_speed_2():
    L, Rt, g = S["secIVA_left"], S["secIVA_right"], S["secIVA_gamma"]["value"]
    left = (L["rho"], L["u"], L["rho"] * L["T"])
    right = (Rt["rho"], Rt["u"], Rt["rho"] * Rt["T"])
    sol = R.solve(left, right, g)
    # the star state is the printed left state (to its rounding): no left-moving wave
    assert abs(sol.p_star - left[2]) <= 2e-5
    assert abs(sol.u_star - left[1]) <= 2e-5
    assert abs(sol.rho_star_left - left[0]) <= 2e-5
    lh, lt, c, rt, rh = sol.wave_speeds()
    assert sol.p_star > right[2] and rt == rh               # the right wave is a shock
    assert abs(rh - 2.0) <= 1e-4
    assert abs(sol.rho_star_right - left[0]) <= 2e-5       # behind it, the shocked density


def test_sec5_pressure_form_and_mach_number():
    s, h = S["secV_shocked"], S["secV_heavy"]
    T_iva = S["secIVA_left"]["T"]
    # p = rho T with R = 1, to the printed rounding of both numbers
    assert abs(s["rho"] * T_iva - s["p"]) <= s["rho"] * _printed_digits_tol(T_iva) + _printed_digits_tol(s["p"])
    # the shock runs at speed 2 into the heavy medium (Sec. IV.A's same state)
    sol = R.solve((s["rho"], s["u"], s["p"]), (h["rho"], h["u"], h["p"]), 2.0)
    speed = sol.wave_speeds()[4]
    mach = speed / math.sqrt(2.0 * h["p"] / h["rho"])
    assert abs(mach - S["secV_mach"]["value"]) <= _printed_digits_tol(S["secV_mach"]["value"])


def test_workloads_transcribe_the_printed_states():
    p = wl.discontinuity(nx=40)
    L, Rt = S["secIVA_left"], S["secIVA_right"]
    left = (p.rho[0, 0], p.ux[0, 0], p.uy[0, 0], p.T[0, 0])
    right = (p.rho[0, -1], p.ux[0, -1], p.uy[0, -1], p.T[0, -1])
    for got, (k, want) in zip(left, L.items()):
        assert abs(got - want) <= _printed_digits_tol(want), k
    for got, (k, want) in zip(right, Rt.items()):
        assert abs(got - want) <= _printed_digits_tol(want), k
    assert p.gamma == S["secIVA_gamma"]["value"]
    q = wl.lax(nx=40)
    L, Rt = S["secIVB_left"], S["secIVB_right"]
    assert (q.rho[0, 0], q.ux[0, 0], q.uy[0, 0], q.T[0, 0]) == (L["rho"], L["u"], L["v"], L["T"])
    assert (q.rho[0, -1], q.ux[0, -1], q.uy[0, -1], q.T[0, -1]) == (Rt["rho"], Rt["u"], Rt["v"], Rt["T"])
    r = wl.shock_heavy_light(nx=1200, ny=10)
    xs = (np.arange(r.nx) + 0.5) * r.dx
    sh, hv, li = S["secV_shocked"], S["secV_heavy"], S["secV_light"]
    for x, st in ((0.1, sh), (0.3, hv), (0.8, li)):
        i = int(np.argmin(np.abs(xs - x)))
        got = (r.rho[0, i], r.ux[0, i], r.uy[0, i], r.rho[0, i] * r.T[0, i])
        for g_, (k, want) in zip(got, st.items()):
            tol = _printed_digits_tol(want)
            if k == "p" and st is sh:
                # printed as 1.5 x 1.55556 (the rounded rho T), not as 7/3 rounded (reading A12)
                tol = st["rho"] * _printed_digits_tol(S["secIVA_left"]["T"]) + tol
            assert abs(g_ - want) <= tol, (x, k)
