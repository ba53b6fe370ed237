"""Closed forms that pin the oracle.

TEST INFRASTRUCTURE ONLY.  R = 1 throughout (so P = rho T).

- Transport coefficients of the recovered Navier-Stokes equations (Sec. II):
  mu = rho R T / s5, lambda' = rho R T / s8, lambda = (b/2 + 1) R lambda',
  hence Pr = mu c_p / lambda = s8 / s5 with c_p = (b + 2) R / 2.
- Thermal Couette profile (Sec. IV.C): T = T1 + (T2 - T1) xi + mu/(2 lambda)
  U^2 xi (1 - xi), xi = distance from the resting wall / H, and mu/(2 lambda)
  = Pr / ((b + 2) R).
- Normal-shock (Rankine-Hugoniot) states of a shock moving at Mach Ma into
  gas at rest.
"""
from __future__ import annotations

import math


def b_of_gamma(gamma: float) -> float:
    """gamma = (b + 2) / b  (Sec. II)."""
    return 2.0 / (gamma - 1.0)


def kinematic_viscosity(T: float, s5: float, rho: float = 1.0) -> float:
    """mu / rho with mu = rho R T / s5."""
    return T / s5


def thermal_diffusivity(T: float, s8: float, b: float, rho: float = 1.0) -> float:
    """lambda / (rho c_p) with lambda = (b/2 + 1) rho R T / s8 and c_p = (b + 2) R / 2."""
    lam = (b / 2.0 + 1.0) * rho * T / s8
    cp = (b + 2.0) / 2.0
    return lam / (rho * cp)


def couette_profile(xi, U: float, Pr: float, b: float, T1: float = 1.0, T2: float = 1.0):
    """Steady thermal Couette flow: (u, T) at xi in [0, 1] (resting wall at xi = 0)."""
    import numpy as np
    xi = np.asarray(xi, dtype=np.float64)
    u = U * xi
    T = T1 + (T2 - T1) * xi + Pr / (b + 2.0) * U * U * xi * (1.0 - xi)
    return u, T


def normal_shock(rho1: float, p1: float, mach: float, gamma: float):
    """State behind a shock moving at Mach `mach` into gas (rho1, 0, p1).

    Returns (rho2, u2, p2, shock_speed)."""
    g, M2 = gamma, mach * mach
    a1 = math.sqrt(g * p1 / rho1)
    S = mach * a1
    rho2 = rho1 * (g + 1.0) * M2 / ((g - 1.0) * M2 + 2.0)
    p2 = p1 * (1.0 + 2.0 * g / (g + 1.0) * (M2 - 1.0))
    u2 = S * (1.0 - rho1 / rho2)
    return rho2, u2, p2, S
