"""Exact solution of the one-dimensional Riemann problem for an ideal gas.

TEST INFRASTRUCTURE ONLY.  Used to pin the shock-tube runs of Sec. IV.A and
IV.B (and the Sod configuration) against the exact Euler solution.

Method (the standard exact solver for the Euler equations of a polytropic
gas): the star pressure p* is the root of f_L(p) + f_R(p) + (u_R - u_L) = 0,
where f_K is the velocity jump across a shock (Rankine-Hugoniot) when
p > p_K and across a rarefaction (isentropic, Riemann invariant) otherwise;
u* follows from f_L, f_R; the solution is self-similar in xi = x/t and is
sampled wave by wave.  R = 1, so p = rho T.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.optimize import brentq


@dataclass
class RiemannSolution:
    gamma: float
    left: tuple      # (rho, u, p)
    right: tuple
    p_star: float
    u_star: float
    rho_star_left: float
    rho_star_right: float

    def wave_speeds(self):
        """(left wave head, left wave tail, contact, right wave tail, right wave head)."""
        g = self.gamma
        rl, ul, pl = self.left
        rr, ur, pr = self.right
        al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
        if self.p_star > pl:
            s = ul - al * math.sqrt((g + 1) / (2 * g) * self.p_star / pl + (g - 1) / (2 * g))
            lh = lt = s
        else:
            lh = ul - al
            lt = self.u_star - al * (self.p_star / pl) ** ((g - 1) / (2 * g))
        if self.p_star > pr:
            s = ur + ar * math.sqrt((g + 1) / (2 * g) * self.p_star / pr + (g - 1) / (2 * g))
            rh = rt = s
        else:
            rh = ur + ar
            rt = self.u_star + ar * (self.p_star / pr) ** ((g - 1) / (2 * g))
        return lh, lt, self.u_star, rt, rh

    def sample(self, xi: np.ndarray):
        """Return (rho, u, p) at similarity coordinates xi = (x - x0)/t."""
        xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
        rho = np.empty_like(xi); u = np.empty_like(xi); p = np.empty_like(xi)
        for n, s in enumerate(xi):
            rho[n], u[n], p[n] = self._sample1(float(s))
        return rho, u, p

    def _sample1(self, s):
        g = self.gamma
        rl, ul, pl = self.left
        rr, ur, pr = self.right
        ps, us = self.p_star, self.u_star
        if s <= us:
            al = math.sqrt(g * pl / rl)
            if ps > pl:
                sl = ul - al * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                return (rl, ul, pl) if s <= sl else (self.rho_star_left, us, ps)
            head = ul - al
            tail = us - al * (ps / pl) ** ((g - 1) / (2 * g))
            if s <= head:
                return rl, ul, pl
            if s >= tail:
                return self.rho_star_left, us, ps
            u = 2.0 / (g + 1) * (al + 0.5 * (g - 1) * ul + s)
            a = 2.0 / (g + 1) * (al + 0.5 * (g - 1) * (ul - s))
            return rl * (a / al) ** (2 / (g - 1)), u, pl * (a / al) ** (2 * g / (g - 1))
        ar = math.sqrt(g * pr / rr)
        if ps > pr:
            sr = ur + ar * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
            return (rr, ur, pr) if s >= sr else (self.rho_star_right, us, ps)
        head = ur + ar
        tail = us + ar * (ps / pr) ** ((g - 1) / (2 * g))
        if s >= head:
            return rr, ur, pr
        if s <= tail:
            return self.rho_star_right, us, ps
        u = 2.0 / (g + 1) * (-ar + 0.5 * (g - 1) * ur + s)
        a = 2.0 / (g + 1) * (ar - 0.5 * (g - 1) * (ur - s))
        return rr * (a / ar) ** (2 / (g - 1)), u, pr * (a / ar) ** (2 * g / (g - 1))


def _f_side(p, rho, pk, g):
    a = math.sqrt(g * pk / rho)
    if p > pk:
        A = 2.0 / ((g + 1) * rho)
        B = (g - 1) / (g + 1) * pk
        return (p - pk) * math.sqrt(A / (p + B))
    return 2.0 * a / (g - 1) * ((p / pk) ** ((g - 1) / (2 * g)) - 1.0)


def solve(left, right, gamma) -> RiemannSolution:
    """left/right = (rho, u, p).  Raises if the data generate vacuum."""
    rl, ul, pl = map(float, left)
    rr, ur, pr = map(float, right)
    g = float(gamma)

    def fun(p):
        return _f_side(p, rl, pl, g) + _f_side(p, rr, pr, g) + (ur - ul)

    lo = 1e-14 * max(pl, pr)
    if fun(lo) > 0:
        raise ValueError("Riemann data generate vacuum")
    hi = max(pl, pr)
    while fun(hi) < 0:
        hi *= 2.0
    ps = brentq(fun, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    us = 0.5 * (ul + ur) + 0.5 * (_f_side(ps, rr, pr, g) - _f_side(ps, rl, pl, g))

    def rho_star(rho, pk):
        if ps > pk:
            q = (g - 1) / (g + 1)
            return rho * (ps / pk + q) / (q * ps / pk + 1.0)
        return rho * (ps / pk) ** (1.0 / g)

    return RiemannSolution(g, (rl, ul, pl), (rr, ur, pr), ps, us, rho_star(rl, pl), rho_star(rr, pr))
