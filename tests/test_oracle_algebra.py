"""Pins of the oracle's algebra against what the paper fixes (CPU only).

- the discrete velocity set and eta_i (Sec. II, Fig. 1; Appendix A);
- M M^-1 = I (Appendix A);
- the seven moment relations of the equilibrium (Appendix A), checked by
  direct summation over the 16 velocities, for every tensor component;
- conservation of rho, j, e by the collision term (Eq. 3 with the modified
  S_88 / S_99 of Sec. II);
- the limiter psi(theta) (Sec. III) at its breakpoints;
- Delta* = M*(f - f^eq) (Sec. V, Appendix A) against independently derived
  polynomial shifts of Delta.
"""
import math

import numpy as np
import pytest

RNG = np.random.default_rng(20130520)


def _states(n):
    """Random (rho, ux, uy, T, b) in the ranges rho in [0.1, 8], |u| <= 0.5, T in [0.25, 4]."""
    out = []
    for k in range(n):
        rho = RNG.uniform(0.1, 8.0)
        ang = RNG.uniform(0, 2 * math.pi)
        mag = RNG.uniform(0, 0.5)
        T = RNG.uniform(0.25, 4.0)
        b = (3.0, 5.0, 10.0)[k % 3]
        out.append((rho, mag * math.cos(ang), mag * math.sin(ang), T, b))
    return out


def test_velocity_set_and_eta(orc):
    _, _, vx, vy, eta = orc.matrices()
    v = {(round(a, 12), round(b, 12)) for a, b in zip(vx, vy)}
    r2 = math.sqrt(2.0)
    expect = set()
    for sx, sy in ((1, 0), (0, 1), (-1, 0), (0, -1)):
        expect.add((float(sx), float(sy)))
        expect.add((6.0 * sx, 6.0 * sy))
    for sx in (1, -1):
        for sy in (1, -1):
            expect.add((round(r2 * sx, 12), round(r2 * sy, 12)))
            expect.add((round(3 / r2 * sx, 12), round(3 / r2 * sy, 12)))
    assert v == expect
    speeds = np.hypot(vx, vy)
    np.testing.assert_allclose(speeds[:4], 1.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(speeds[4:8], 6.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(speeds[8:12], 2.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(speeds[12:], 3.0, rtol=0, atol=1e-15)
    assert np.all(eta[:4] == 2.5) and np.all(eta[4:] == 0.0)


def test_M_times_Minv_is_identity(orc):
    M, Mi, *_ = orc.matrices()
    assert np.abs(M @ Mi - np.eye(16)).max() <= 1e-13
    assert np.abs(Mi @ M - np.eye(16)).max() <= 1e-13


@pytest.mark.parametrize("state", _states(24))
def test_seven_moment_relations(orc, state):
    """Sum_i f_i^eq phi(v_i) reproduces every relation of Appendix A (R = 1)."""
    rho, ux, uy, T, b = state
    _, _, vx, vy, eta = orc.matrices()
    f = orc.feq(rho, ux, uy, T, b)
    P = rho * T
    u = (ux, uy)
    u2 = ux * ux + uy * uy
    v = (vx, vy)
    w = vx * vx + vy * vy + eta * eta
    d = lambda a, c: 1.0 if a == c else 0.0  # noqa: E731
    checks = []
    checks.append((f.sum(), rho))
    for a in range(2):
        checks.append(((f * v[a]).sum(), rho * u[a]))
    checks.append(((f * w).sum(), rho * (b * T + u2)))
    for a in range(2):
        for c in range(a, 2):
            checks.append(((f * v[a] * v[c]).sum(), P * d(a, c) + rho * u[a] * u[c]))
    for a in range(2):
        checks.append(((f * w * v[a]).sum(), rho * ((b + 2) * T + u2) * u[a]))
    for a in range(2):
        for c in range(a, 2):
            for e in range(c, 2):
                lhs = (f * v[a] * v[c] * v[e]).sum()
                rhs = rho * (T * (u[a] * d(c, e) + u[c] * d(a, e) + u[e] * d(a, c)) + u[a] * u[c] * u[e])
                checks.append((lhs, rhs))
    for a in range(2):
        for c in range(a, 2):
            lhs = (f * w * v[a] * v[c]).sum()
            rhs = rho * ((b + 2) * T * T * d(a, c) + ((b + 4) * u[a] * u[c] + u2 * d(a, c)) * T
                         + u2 * u[a] * u[c])
            checks.append((lhs, rhs))
    assert len(checks) == 16
    scale = rho * (1 + T) ** 2 * 40
    for lhs, rhs in checks:
        assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs)


def _random_noneq(orc, rho, ux, uy, T, b, amp=1e-2):
    """f = f^eq(rho, u, T) + a perturbation with zero mass, momentum and energy."""
    _, _, vx, vy, eta = orc.matrices()
    feq = orc.feq(rho, ux, uy, T, b)
    C = np.stack([np.ones(16), vx, vy, vx * vx + vy * vy + eta * eta])  # 4 x 16
    p = RNG.normal(size=16) * amp * rho
    p -= C.T @ np.linalg.solve(C @ C.T, C @ p)
    return feq + p, feq


@pytest.mark.parametrize("state", _states(12))
def test_collision_conserves_mass_momentum_energy(orc, state):
    rho, ux, uy, T, b = state
    gamma = (b + 2) / b
    f, _ = _random_noneq(orc, rho, ux, uy, T, b, amp=5e-2)
    s = RNG.uniform(1e2, 1e4, 16)
    s[4:7] = s[4]
    s[7:9] = s[7]
    grad = RNG.normal(size=4)
    C = orc.collision(f, s, gamma, grad)
    M, _, vx, vy, eta = orc.matrices()
    scale = np.abs(s).max() * np.abs(M @ f).max()
    for phi in (np.ones(16), vx, vy, vx * vx + vy * vy + eta * eta):
        assert abs((C * phi).sum()) <= 1e-14 * scale


def test_collision_vanishes_at_equilibrium(orc):
    for rho, ux, uy, T, b in _states(6):
        f = orc.feq(rho, ux, uy, T, b)
        C = orc.collision(f, np.full(16, 1e3), (b + 2) / b, (0.0, 0.0, 0.0, 0.0))
        assert np.abs(C).max() <= 1e-9 * rho * (1 + T) ** 2


@pytest.mark.parametrize("theta,psi", [(-3.0, 0.0), (-1e-300, 0.0), (0.0, 0.0), (0.1, 0.2),
                                       (1.0 / 3.0, 2.0 / 3.0), (1.0, 1.0), (2.0, 1.5), (3.0, 2.0),
                                       (7.5, 2.0), (1e300, 2.0)])
def test_limiter_psi_breakpoints(orc, theta, psi):
    assert orc.psi(theta) == pytest.approx(psi, rel=1e-15, abs=0)


def test_limiter_psi_continuous_and_bounded(orc):
    th = np.linspace(-2, 6, 8001)
    ps = np.array([orc.psi(t) for t in th])
    assert ps.min() >= 0.0 and ps.max() <= 2.0
    assert np.abs(np.diff(ps)).max() <= 2 * (th[1] - th[0]) + 1e-15
    # TVD region of the (theta, psi) plane: psi <= 2 theta and psi <= 2
    assert np.all(ps <= np.maximum(2 * th, 0) + 1e-15)


def test_central_matrix_reduces_to_M_at_rest(orc):
    M, *_ = orc.matrices()
    assert np.array_equal(orc.central_matrix(0.0, 0.0), M)


@pytest.mark.parametrize("state", _states(9))
def test_delta_star_polynomial_shift(orc, state):
    """Delta* rows against the shift of Delta derived by hand (conserved rows vanish)."""
    rho, ux, uy, T, b = state
    f, feq = _random_noneq(orc, rho, ux, uy, T, b)
    M, *_ = orc.matrices()
    D = M @ (f - feq)                     # Delta (1-based row k is D[k-1])
    Ds = orc.central_matrix(ux, uy) @ (f - feq)
    sc = np.abs(D).max()
    for k in range(4):
        assert abs(Ds[k]) <= 1e-12 * sc
    # second order: unchanged
    for k in (4, 5, 6):
        assert Ds[k] == pytest.approx(D[k], abs=1e-12 * sc)
    # third order, (v_x - u_x)|v - u|^2 = m10 - u_x (2 m5 + m6) - 2 u_y m7 + ...
    d10 = D[9] - ux * (2 * D[4] + D[5]) - 2 * uy * D[6]
    d11 = D[10] - uy * (2 * D[4] - D[5]) - 2 * ux * D[6]
    assert Ds[9] == pytest.approx(d10, abs=1e-11 * sc)
    assert Ds[10] == pytest.approx(d11, abs=1e-11 * sc)
    # eta^2 part: sum delta eta^2 (v - u) = (Delta_8 - Delta_10) + u_x Delta_5 (x); same in y
    assert Ds[7] == pytest.approx(d10 + (D[7] - D[9]) + ux * D[4], abs=1e-11 * sc)
    assert Ds[8] == pytest.approx(d11 + (D[8] - D[10]) + uy * D[4], abs=1e-11 * sc)
    # (v_x - u_x)((v_x-u_x)^2 - (v_y-u_y)^2) = m12 - u_x (m5 + m6) ... expanded by hand
    d12 = D[11] - 3 * ux * (D[4] + D[5]) / 2 + 2 * uy * D[6] + ux * (D[4] - D[5]) / 2
    assert Ds[11] == pytest.approx(d12, abs=1e-11 * sc)
