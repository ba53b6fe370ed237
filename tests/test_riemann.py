"""Pins of the exact Riemann solver used to check the shock-tube runs (CPU only).

The solver is checked against conditions that do not come from its own
formulas: the Rankine-Hugoniot jump conditions across its shocks, the
isentropic relation and Riemann invariant across its rarefactions, and the
paper's discontinuity test (Sec. IV.A), whose two states satisfy the Hugoniot
relations so that the exact solution is a single shock (gamma = 2, speed 2).
"""
import math

import pytest

from oracle import riemann
from oracle.analytic import normal_shock


def _rh_residuals(g, rho1, u1, p1, rho2, u2, p2, S):
    """Mass, momentum and energy fluxes in the shock frame, left minus right."""
    def fluxes(r, u, p):
        w = u - S
        E = p / (g - 1) + 0.5 * r * w * w
        return r * w, r * w * w + p, (E + p) * w
    a, b = fluxes(rho1, u1, p1), fluxes(rho2, u2, p2)
    return [abs(x - y) for x, y in zip(a, b)]


def test_paper_discontinuity_states_give_a_single_shock():
    # Sec. IV.A: (1.5, 0.666667, 0, T = 1.55556) | (1, 0, 0, 1), gamma = 2; exact values 2/3, 14/9
    left = (1.5, 2.0 / 3.0, 1.5 * 14.0 / 9.0)
    right = (1.0, 0.0, 1.0)
    sol = riemann.solve(left, right, 2.0)
    assert sol.p_star == pytest.approx(7.0 / 3.0, rel=1e-12)
    assert sol.u_star == pytest.approx(2.0 / 3.0, rel=1e-12)
    assert sol.rho_star_left == pytest.approx(1.5, rel=1e-12)
    assert sol.rho_star_right == pytest.approx(1.5, rel=1e-12)
    *_, rt, rh = sol.wave_speeds()
    assert rt == rh == pytest.approx(2.0, rel=1e-12)
    # and the paper's rounded decimals are those of a Mach sqrt(2) shock into (1, 0, 1)
    r2, u2, p2, S = normal_shock(1.0, 1.0, math.sqrt(2.0), 2.0)
    assert (r2, u2, p2, S) == pytest.approx((1.5, 2.0 / 3.0, 7.0 / 3.0, 2.0), rel=1e-12)
    assert round(u2, 6) == 0.666667 and round(p2 / r2, 5) == 1.55556


@pytest.mark.parametrize("left,right,g", [((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4),
                                          ((0.445, 0.698, 0.445 * 7.928), (0.5, 0.0, 0.5 * 1.142), 1.4),
                                          ((1.0, 0.0, 1000.0), (1.0, 0.0, 0.01), 1.4),
                                          ((2.0, 0.3, 3.0), (1.0, -0.2, 0.5), 5.0 / 3.0)])
def test_jump_conditions(left, right, g):
    sol = riemann.solve(left, right, g)
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = sol.p_star, sol.u_star
    # right wave
    if ps > pr:
        S = sol.wave_speeds()[4]
        res = _rh_residuals(g, sol.rho_star_right, us, ps, rr, ur, pr, S)
        assert max(res) <= 1e-10 * max(1.0, ps)
    else:
        assert ps / sol.rho_star_right ** g == pytest.approx(pr / rr ** g, rel=1e-12)
        a_s = math.sqrt(g * ps / sol.rho_star_right)
        ar = math.sqrt(g * pr / rr)
        assert us - 2 * a_s / (g - 1) == pytest.approx(ur - 2 * ar / (g - 1), rel=1e-12, abs=1e-12)
    # left wave
    if ps > pl:
        S = sol.wave_speeds()[0]
        res = _rh_residuals(g, rl, ul, pl, sol.rho_star_left, us, ps, S)
        assert max(res) <= 1e-10 * max(1.0, ps)
    else:
        assert ps / sol.rho_star_left ** g == pytest.approx(pl / rl ** g, rel=1e-12)
        a_s = math.sqrt(g * ps / sol.rho_star_left)
        al = math.sqrt(g * pl / rl)
        assert us + 2 * a_s / (g - 1) == pytest.approx(ul + 2 * al / (g - 1), rel=1e-12)


def test_fan_is_continuous():
    sol = riemann.solve((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
    lh, lt, *_ = sol.wave_speeds()
    import numpy as np
    xi = np.linspace(lh - 1e-9, lt + 1e-9, 2001)
    r, u, p = sol.sample(xi)
    assert np.abs(np.diff(r)).max() < 2e-3 and np.abs(np.diff(p)).max() < 2e-3
    assert r[0] == pytest.approx(1.0) and r[-1] == pytest.approx(sol.rho_star_left)
