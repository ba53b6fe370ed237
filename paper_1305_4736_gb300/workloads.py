"""Seeded synthetic inputs: problem parameters and initial macroscopic fields.

This module holds no arithmetic of the lattice Boltzmann method: it only lays
out initial density, velocity and temperature fields and the run parameters
(grid, time step, relaxation rates, boundary kinds) of the shock-tube,
Couette, shock-interface, shear-layer and serving workloads.  Both the GPU
library and the CPU oracle consume what it returns.

Conventions: cell-centred grid, x_i = (i + 1/2) dx, y_j = (j + 1/2) dy;
fields are float64 arrays [ny][nx]; R = 1, so T = p / rho.  Relaxation rates
are s_1..s_16 (s_1..s_4 belong to conserved moments and are unused).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Boundary kinds and limiter ids (same values as the C interface).
BC_PERIODIC, BC_ZERO_GRADIENT, BC_EQUILIBRIUM, BC_NEQ_WALL = 0, 1, 2, 3
LIMITER_MC, LIMITER_LW, LIMITER_UPWIND = 0, 1, 2
FP64, FP32_DEV = 0, 1

SEED = 1305


@dataclass
class Problem:
    name: str
    nx: int
    ny: int
    dx: float
    dt: float
    gamma: float
    Pr: float
    s: np.ndarray                       # 16 relaxation rates
    bc: list                            # 4 x (kind, rho, ux, uy, T): x-lo, x-hi, y-lo, y-hi
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    T: np.ndarray
    steps: int
    limiter: int = LIMITER_MC
    meta: dict = field(default_factory=dict)
    dy: float | None = None             # grid spacing along y; None: dy = dx

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def fields(self):
        return self.rho, self.ux, self.uy, self.T


def rates(s5: float, s8: float | None = None, others: float | None = None) -> np.ndarray:
    """s_5 = s_6 = s_7 = s5, s_8 = s_9 = s8 (default s5), all other rates `others` (default s5)."""
    s8 = s5 if s8 is None else s8
    others = s5 if others is None else others
    s = np.full(16, float(others))
    s[4:7] = s5
    s[7:9] = s8
    return s


def periodic_bc():
    return [(BC_PERIODIC, 0.0, 0.0, 0.0, 0.0)] * 4


def _centres(n: int, d: float) -> np.ndarray:
    return (np.arange(n) + 0.5) * d


def normal_shock_state(rho1: float, p1: float, mach: float, gamma: float):
    """Gas-dynamics input preparation: post-shock (rho, u, p) and shock speed of a
    shock moving at `mach` into gas at rest (Rankine-Hugoniot relations)."""
    g, m2 = gamma, mach * mach
    speed = mach * math.sqrt(g * p1 / rho1)
    rho2 = rho1 * (g + 1.0) * m2 / ((g - 1.0) * m2 + 2.0)
    p2 = p1 * (1.0 + 2.0 * g / (g + 1.0) * (m2 - 1.0))
    return rho2, speed * (1.0 - rho1 / rho2), p2, speed


def riemann(nx: int = 200, ny: int = 4, left=(1.0, 0.0, 0.0, 1.0), right=(0.125, 0.0, 0.0, 0.8),
            gamma: float = 1.4, s: float | np.ndarray = 5e3, length: float = 1.0,
            dt: float | None = None, t_end: float = 0.2, limiter: int = LIMITER_MC,
            name: str = "riemann", bc_kind: int = BC_ZERO_GRADIENT) -> Problem:
    """Shock tube along x: left/right = (rho, u, v, T), discontinuity at length/2.
    Defaults are the Sod tube of 200 x 4 cells, dx = 5e-3, dt = 1e-4, 2000 steps."""
    dx = length / nx
    if dt is None:
        dt = 1e-4 * (dx / 5e-3)
    x = _centres(nx, dx)
    left_mask = np.broadcast_to(x < 0.5 * length, (ny, nx))
    f = [np.where(left_mask, left[k], right[k]).astype(np.float64) for k in range(4)]
    sr = rates(s) if np.isscalar(s) else np.asarray(s, dtype=np.float64)
    if bc_kind == BC_EQUILIBRIUM:
        xlo = (BC_EQUILIBRIUM,) + tuple(float(v) for v in left)
        xhi = (BC_EQUILIBRIUM,) + tuple(float(v) for v in right)
    else:
        xlo = xhi = (bc_kind, 0.0, 0.0, 0.0, 0.0)
    bc = [xlo, xhi, (BC_PERIODIC, 0, 0, 0, 0), (BC_PERIODIC, 0, 0, 0, 0)]
    steps = int(round(t_end / dt))
    return Problem(name, nx, ny, dx, dt, gamma, float(sr[7] / sr[4]), sr, bc,
                   np.ascontiguousarray(f[0]), np.ascontiguousarray(f[1]),
                   np.ascontiguousarray(f[2]), np.ascontiguousarray(f[3]), steps, limiter,
                   {"left": left, "right": right, "length": length, "t_end": t_end})


def sod(nx: int = 200, ny: int = 4, steps: int | None = None) -> Problem:
    """Sod shock tube: rho = 1, T = 1 | rho = 0.125, T = 0.8; gamma = 1.4; all s = 5e3;
    200 x 4 cells, dx = 5e-3, dt = 1e-4, 2000 steps (t = 0.2); zero-gradient x ends."""
    p = riemann(nx, ny, name="sod")
    if steps is not None:
        p.steps = steps
    return p


def discontinuity(nx: int = 1000, ny: int = 4, limiter: int = LIMITER_MC) -> Problem:
    """The discontinuity test of Sec. IV.A at the paper's parameters: gamma = 2,
    (rho, u, v, T) = (3/2, 2/3, 0, 14/9) | (1, 0, 0, 1) (the Hugoniot states of a Mach-sqrt2
    shock moving at speed 2 into gas at rest; the paper prints them rounded), L = 1, dx = dy =
    1e-3, dt = 1e-5, s5 = s6 = s7 = 5e4 and every other rate 1e5 (so s8 = s9 = 1e5), fixed
    equilibrium x ends, periodic y, t = 0.06 (6000 steps)."""
    r2, u2, p2, _ = normal_shock_state(1.0, 1.0, math.sqrt(2.0), 2.0)
    p = riemann(nx, ny, (r2, u2, 0.0, p2 / r2), (1.0, 0.0, 0.0, 1.0), 2.0, rates(5e4, 1e5, 1e5),
                length=nx * 1e-3, dt=1e-5, t_end=0.06, limiter=limiter, name="discontinuity",
                bc_kind=BC_EQUILIBRIUM)
    return p


def lax(nx: int = 1000, ny: int = 4, limiter: int = LIMITER_MC) -> Problem:
    """The Lax shock tube of Sec. IV.B at the paper's parameters: gamma = 1.4,
    (rho, u, v, T) = (0.445, 0.698, 0, 7.928) | (0.5, 0, 0, 1.142), dx = dy = 3e-3, dt = 1e-5,
    s5 = s6 = s7 = 2e3, s8 = s9 = 1e3, other rates 1e5, t = 0.45 (45000 steps).  The paper does
    not give L; 1000 cells (L = 3, diaphragm at 1.5) keep every wave inside until t = 0.45.
    Fixed equilibrium x ends, periodic y."""
    return riemann(nx, ny, (0.445, 0.698, 0.0, 7.928), (0.5, 0.0, 0.0, 1.142), 1.4, rates(2e3, 1e3, 1e5),
                   length=nx * 3e-3, dt=1e-5, t_end=0.45, limiter=limiter, name="lax", bc_kind=BC_EQUILIBRIUM)


def couette(Pr: float = 1.0, nx: int = 4, ny: int = 200, dx: float | None = None,
            dt: float | None = None, u0: float = 0.2, gamma: float = 1.4, s5: float = 1e3,
            T_low: float = 1.0, T_high: float = 1.0, steps: int = 1000) -> Problem:
    """Thermal Couette flow between walls at y = 0 (rest, T_low) and y = H = 1 (moving at u0
    along x, T_high); periodic x; rho = 1, u = 0, T = 1 initially.
    s_5..7 = s5, s_8..9 = Pr s5, others s5 (the paper's (s5, s8) pairing, Sec. IV.C)."""
    dx = (1.0 / ny) if dx is None else dx
    dt = (5e-5 * (dx / 5e-3)) if dt is None else dt
    one = np.ones((ny, nx))
    bc = [(BC_PERIODIC, 0, 0, 0, 0), (BC_PERIODIC, 0, 0, 0, 0),
          (BC_NEQ_WALL, 1.0, 0.0, 0.0, T_low), (BC_NEQ_WALL, 1.0, u0, 0.0, T_high)]
    s = rates(s5, Pr * s5, s5)
    return Problem("couette", nx, ny, dx, dt, gamma, Pr, s, bc, one.copy(), 0.0 * one,
                   0.0 * one, one.copy(), steps, LIMITER_MC, {"u0": u0, "H": ny * dx})


def shock_interface(nx: int = 4096, ny: int = 1024, seed: int = SEED, steps: int = 5000,
                    p0: float = 2.0) -> Problem:
    """Mach-1.5 shock in heavy gas (rho = 4, p = p0) hitting a light gas (rho = 1, p = p0)
    across a sinusoidal interface x_i(y) = 0.6 Lx/4 + 0.02 Ly cos(2 pi y/Ly + phi), phi seeded.
    Lx = 4 Ly, Ly = 1, dx = Ly/ny, dt = 5e-5 (s dt = 0.5 at every size); gamma = 1.4, all s = 1e4;
    x-lo fixed equilibrium (post-shock), x-hi zero-gradient, periodic y.
    p0 = 2 (T = 0.5 in the heavy gas, 2 in the light gas): at p0 = 1 (T = 0.25) the full-size
    run (dx = 1/1024, Courant 0.31) goes non-finite about 1300 steps after the shock meets the
    interface (step ~3600 of 5000; the equilibria are strongly negative at T = 0.25)."""
    gamma = 1.4
    Lx, Ly = 4.0 * (nx / (4 * ny)), 1.0
    dx = Ly / ny
    dt = 5e-5
    phi = np.random.default_rng(seed).uniform(0.0, 2.0 * math.pi)
    rho_s, u_s, p_s, speed = normal_shock_state(4.0, p0, 1.5, gamma)
    x = _centres(nx, dx)[None, :]
    y = _centres(ny, dx)[:, None]
    x_shock, x_if = 0.5, 0.6 + 0.02 * Ly * np.cos(2 * math.pi * y / Ly + phi)
    rho = np.where(x < x_shock, rho_s, np.where(x < x_if, 4.0, 1.0))
    p = np.where(x < x_shock, p_s, p0) * np.ones_like(rho)
    ux = np.where(x < x_shock, u_s, 0.0) * np.ones_like(rho)
    T = p / rho
    bc = [(BC_EQUILIBRIUM, rho_s, u_s, 0.0, p_s / rho_s), (BC_ZERO_GRADIENT, 0, 0, 0, 0),
          (BC_PERIODIC, 0, 0, 0, 0), (BC_PERIODIC, 0, 0, 0, 0)]
    s = rates(1e4)
    return Problem("shock_interface", nx, ny, dx, dt, gamma, 1.0, s, bc,
                   np.ascontiguousarray(rho), np.ascontiguousarray(ux),
                   np.zeros_like(rho), np.ascontiguousarray(T), steps, LIMITER_MC,
                   {"phi": phi, "shock_speed": speed, "Lx": Lx, "Ly": Ly})


def shear_layer(n: int = 8192, seed: int = SEED, steps: int = 2000, ny: int | None = None) -> Problem:
    """Doubly periodic low-Mach double shear layer on the unit square: rho = 1, T = 1,
    u_x = 0.05 tanh((y - 1/4)/delta) for y < 1/2 and 0.05 tanh((3/4 - y)/delta) above,
    delta = 1/160; v = seeded 8-mode sine perturbation rescaled to max |v| = 1e-3.
    gamma = 1.4, Pr = 0.71: s_5..7 = 5e4, s_8..9 = 3.55e4, others 1e5; dx = 1/n,
    dt = min(1e-5, dx/24): 1e-5 up to n = 2400 (s dt <= 1), and a largest Courant number of
    1/4 above (n = 8192: dt = 5.09e-6, s dt <= 0.51).  At n = 8192 and dt = 1e-5 (Courant
    0.49, s dt = 1 for the fastest moments) the MC-limited step is unstable: grid-scale noise
    grows to overflow within a few hundred steps.  `ny` (default n) allows rectangular test
    grids with the same dx."""
    nx = n
    ny = n if ny is None else ny
    dx = 1.0 / n
    dt = min(1e-5, dx / 24.0)
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, 1.0, 8)
    ph = rng.uniform(0.0, 2.0 * math.pi, 8)
    x = _centres(nx, dx)
    y = _centres(ny, dx)
    delta = 1.0 / 160.0
    ux_col = np.where(y < 0.5, 0.05 * np.tanh((y - 0.25) / delta), 0.05 * np.tanh((0.75 - y) / delta))
    k = np.arange(1, 9)[:, None]
    v_row = (a[:, None] * np.sin(2 * math.pi * k * x[None, :] + ph[:, None])).sum(axis=0)
    v_row *= 1e-3 / np.max(np.abs(v_row))
    ux = np.ascontiguousarray(np.broadcast_to(ux_col[:, None], (ny, nx)))
    uy = np.ascontiguousarray(np.broadcast_to(v_row[None, :], (ny, nx)))
    one = np.ones((ny, nx))
    s = rates(5e4, 3.55e4, 1e5)
    return Problem("shear_layer", nx, ny, dx, dt, 1.4, 0.71, s, periodic_bc(), one, ux, uy,
                   one.copy(), steps, LIMITER_MC, {"delta": delta})


def serving_requests(count: int = 512, seed: int = SEED, rate_hz: float = 100.0,
                     max_nx: int = 2048, max_ny: int = 512, steps: int = 1000):
    """Seeded mixed request stream: 1/3 Riemann, 1/3 Couette, 1/3 shock-interface;
    nx log-uniform in [64, max_nx], ny log-uniform in [4, max_ny] (Couette channels at least
    16 cells wide); gamma in [1.25, 1.5], Pr in [0.5, 2]; FP32/FP64 50/50; Poisson arrival
    times at `rate_hz`.  dt gives a largest Courant number of 0.12 and every s dt <= 0.5
    (the ratios of the Sod configuration); Riemann requests take s dt <= 0.25, since at 0.5 a
    strong rarefaction into a light, cold gas (rho = 0.11, T = 0.55 against 0.88, 1.37 at
    Pr = 1.78) diverged by t = 0.22 whatever the time step, in the oracle as on the GPU.
    Outside gamma in [1.25, 1.5] the discrete-velocity model itself is linearly unstable at
    these rates (see the design notes), and a Courant number of 0.3 let narrow channels
    diverge.
    Returns a list of dicts {kind, arrival, problem, precision}."""
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    for i in range(count):
        t += rng.exponential(1.0 / rate_hz)
        nx = int(round(math.exp(rng.uniform(math.log(64), math.log(max_nx)))))
        ny = int(round(math.exp(rng.uniform(math.log(4), math.log(max_ny)))))
        gamma = float(rng.uniform(1.25, 1.5))
        Pr = float(rng.uniform(0.5, 2.0))
        kind = ("riemann", "couette", "shock_interface")[i % 3]
        precision = FP64 if rng.uniform() < 0.5 else FP32_DEV
        dt_fn = lambda d: 0.12 * d / 6.0                    # largest Courant number 0.12
        if kind == "riemann":
            rl, rr = rng.uniform(0.1, 1.0, 2)
            tl, tr = rng.uniform(0.5, 1.5, 2)
            dt = dt_fn(1.0 / nx)
            s5 = 0.25 / dt / max(1.0, Pr)                      # s dt <= 0.25 for every rate
            prob = riemann(nx, ny, (rl, 0.0, 0.0, tl), (rr, 0.0, 0.0, tr), gamma,
                           rates(s5, Pr * s5, 0.25 / dt), dt=dt, t_end=steps * dt)
        elif kind == "couette":
            u0 = float(rng.uniform(0.05, 0.3))
            ny = max(ny, 16)
            dt = dt_fn(1.0 / ny)
            s5 = 0.5 / dt / max(1.0, Pr)
            prob = couette(Pr, nx=nx, ny=ny, dt=dt, u0=u0, gamma=gamma, s5=s5, steps=steps)
        else:
            prob = shock_interface(nx=max(nx, 8), ny=ny, seed=int(rng.integers(1 << 30)), steps=steps)
            prob.dt = dt_fn(prob.dx)
            prob.s = rates(0.5 / prob.dt)
        prob.steps = steps
        out.append({"id": i, "kind": kind, "arrival": t, "problem": prob, "precision": precision})
    return out


def shock_heavy_light(nx: int = 1200, ny: int = 10, steps: int = 30000) -> Problem:
    """Shock travelling from a heavy into a light medium (the non-equilibrium study of Sec. V):
    domain [0, 1.2] x [0, 0.01] on 1200 x 10 cells; shocked gas (1.5, 2/3, 0, p = 7/3) left of
    x = 0.24, heavy gas (1, 0, 0, p = 1) up to the interface at x = 0.4, light gas (0.5, 0, 0, p = 1)
    beyond; gamma = 2; inflow (fixed shocked equilibrium) on the left, outflow (zero gradient) on
    the right, periodic y; dt = 1e-5, s_5..7 = 5e4, others 1e5; 30000 steps (t = 0.3).
    The paper's rounded states 0.666667 and 2.33334 are taken as the exact Rankine-Hugoniot values."""
    gamma = 2.0
    dx = 1.2 / nx
    rho_s, u_s, p_s, speed = normal_shock_state(1.0, 1.0, math.sqrt(2.0), gamma)
    x = _centres(nx, dx)[None, :] * np.ones((ny, 1))
    rho = np.where(x < 0.24, rho_s, np.where(x < 0.4, 1.0, 0.5))
    p = np.where(x < 0.24, p_s, 1.0)
    ux = np.where(x < 0.24, u_s, 0.0)
    bc = [(BC_EQUILIBRIUM, rho_s, u_s, 0.0, p_s / rho_s), (BC_ZERO_GRADIENT, 0, 0, 0, 0),
          (BC_PERIODIC, 0, 0, 0, 0), (BC_PERIODIC, 0, 0, 0, 0)]
    s = rates(5e4, 5e4, 1e5)
    return Problem("shock_heavy_light", nx, ny, dx, 1e-5, gamma, 1.0, s, bc,
                   np.ascontiguousarray(rho), np.ascontiguousarray(ux), np.zeros((ny, nx)),
                   np.ascontiguousarray(p / rho), steps, LIMITER_MC,
                   {"x_shock": 0.24, "x_interface": 0.4, "shock_speed": speed,
                    "shocked": (rho_s, u_s, p_s), "heavy": (1.0, 0.0, 1.0), "light": (0.5, 0.0, 1.0)})
