"""Pin of the energy-flux correction (Sec. II, modified S_88 and S_99) on a mean flow.

Row 8 of M is v_x (v^2 + eta^2) and row 9 is v_y (v^2 + eta^2): the x and y
fluxes of row 4 (e, twice the total energy).  Their non-equilibrium parts
Delta_8 = f^_8 - f^_8^eq and Delta_9 are therefore the dissipative energy flux,
and the corrected energy equation of Sec. II fixes them at first
Chapman-Enskog order (R = 1, P = rho T, s8 = s9, s5 = s6 = s7):

    Delta_8 = -2 P [ (b/2 + 1) dT/dx / s8 + W_x / s5 ]
    Delta_9 = -2 P [ (b/2 + 1) dT/dy / s9 + W_y / s5 ]
    W_x = (2 du_x/dx - (2/b) div u) u_x + (du_y/dx + du_x/dy) u_y
    W_y = (du_y/dx + du_x/dy) u_x + (2 du_y/dy - (2/b) div u) u_y

Without the correction the W terms would carry 1/s8 instead of 1/s5.  About a
uniform mean flow U every W term is linear in the perturbation (U times a
velocity gradient), so a small wave on U makes each printed coefficient of the
correction visible separately:

- a wave along x on U = (Ux, Uy) gives, in Delta_8, the dT/dx term, Ux du_x/dx
  (the 4 - 4/b of row 8) and Uy du_y/dx (the 2 du_y/dx of row 8); in Delta_9,
  Ux du_y/dx (row 9's 2 du_y/dx) and Uy du_x/dx (row 9's -4/b du_x/dx);
- a wave along y gives the mirror images: Ux du_y/dy (row 8's -4/b du_y/dy),
  Uy du_x/dy, the dT/dy term, Uy du_y/dy and Ux du_x/dy.

The test fits the oracle's Delta_8 and Delta_9 (complex Fourier amplitudes at
the wave number, sampled over a third of a time unit so that the acoustic,
shear and entropy parts of the wave pass through different phases) on those
terms, one coefficient per term, and requires each coefficient to be 1.  The
first-order relation has O(1/s) corrections (a relaxation lag and Burnett
terms: 20% on the smallest term at s5 = 2000); a Richardson step over
s5 = 4000 and 16000 removes them.  What remains is the second-order central
difference of the scheme, a factor sin(kh)/(kh) = 1 - (kh)^2/6 = 0.9984 at
64 cells per wavelength, common to every term.  The Lax-Wendroff limiter
(psi = 1) keeps the scheme linear, so no limiter clipping adds numerical
diffusion to the non-equilibrium parts.

Planting any one of these mistakes in a copy of the oracle moves at least one
coefficient by 12% or more: 4/b -> 2/b in either -4/b term of row 8 or row 9,
4 du_x/dx -> 2 du_x/dx or dropped, 4 du_y/dy -> 2 du_y/dy in row 9, either
2 du/dx or 2 du/dy shear term halved or dropped, -4/b du_y/dy -> +4 du_y/dy,
and the whole correction removed.
"""
import math

import numpy as np
import pytest

from paper_1305_4736_gb300 import workloads as wl

N = 64                  # cells per wavelength (one wavelength over the unit domain)
K = 2.0 * math.pi
U = (0.3, 0.2)          # mean flow (Mach 0.3)
A = 1e-4                # perturbation amplitude
GAMMA = 1.4


def _fit(orc, axis, Pr, s5):
    """Fitted coefficients of the Delta_8 and Delta_9 terms for one run."""
    b = 2.0 / (GAMMA - 1.0)
    s8 = Pr * s5
    other = 2.0 * s5
    dt = 0.2 / other                      # s dt = 0.2 for the fastest moments
    every = int(round(0.02 / dt))         # 15 samples over t = 0.3
    h = 1.0 / N
    shape = (1, N) if axis == 0 else (N, 1)
    phase = (K * (np.arange(N) + 0.5) * h).reshape(shape)
    dux = A * np.cos(phase)               # acoustic + shear + entropy parts, distinct phases
    duy = 0.7 * A * np.sin(phase)
    dT = 0.5 * A * np.cos(phase + 1.0)
    nx, ny = (N, 1) if axis == 0 else (1, N)
    O = orc.Oracle(nx, ny, h, dt, GAMMA, wl.rates(s5, s8, other), orc.LIM_LW, wl.periodic_bc())
    O.init(1.0, U[0] + dux, U[1] + duy, 1.0 + dT)

    def amp(a):
        return 2.0 * np.mean((a - a.mean()) * np.exp(-1j * phase))

    ik = 1j * K
    X8, X9, Y8, Y9 = [], [], [], []
    for _ in range(15):
        O.step(every)
        rho, ux, uy, T, D = O.moments(delta=True)
        P = float(np.mean(rho * T))
        gu, gv, gT = ik * amp(ux), ik * amp(uy), ik * amp(T)
        if axis == 0:
            dxux, dxuy, dxT, dyux, dyuy, dyT = gu, gv, gT, 0.0, 0.0, 0.0
        else:
            dxux, dxuy, dxT, dyux, dyuy, dyT = 0.0, 0.0, 0.0, gu, gv, gT
        heat, work = -2.0 * P * (b / 2.0 + 1.0) / s8, -2.0 * P / s5
        X8.append([heat * dxT, work * U[0] * (2.0 - 2.0 / b) * dxux, work * U[0] * (-2.0 / b) * dyuy,
                   work * U[1] * dxuy, work * U[1] * dyux])
        X9.append([heat * dyT, work * U[1] * (2.0 - 2.0 / b) * dyuy, work * U[1] * (-2.0 / b) * dxux,
                   work * U[0] * dxuy, work * U[0] * dyux])
        Y8.append(amp(D[7]))
        Y9.append(amp(D[8]))
    out = {}
    for row, X, Y in (("Delta8", X8, Y8), ("Delta9", X9, Y9)):
        X = np.array(X, dtype=complex)
        Y = np.array(Y, dtype=complex)
        cols = [j for j in range(X.shape[1]) if np.abs(X[:, j]).max() > 0]
        Xr = np.concatenate([X[:, cols].real, X[:, cols].imag])
        Yr = np.concatenate([Y.real, Y.imag])
        coef = np.linalg.lstsq(Xr, Yr, rcond=None)[0]
        out.update({(row, j): c for j, c in zip(cols, coef)})
    return out


TERMS = {0: "heat flux", 1: "U_a (2 - 2/b) du_a/da", 2: "U_a (-2/b) du_b/db",
         3: "U_b du_b/da", 4: "U_b du_a/db"}


@pytest.mark.parametrize("Pr", [0.5, 2.0])
@pytest.mark.parametrize("axis", [0, 1], ids=["x-wave", "y-wave"])
def test_energy_flux_correction_on_mean_flow(orc, axis, Pr):
    lo = _fit(orc, axis, Pr, 4000.0)
    hi = _fit(orc, axis, Pr, 16000.0)
    assert lo.keys() == hi.keys() and len(lo) == 5          # 3 terms in one row, 2 in the other
    for key in lo:
        c = (4.0 * hi[key] - lo[key]) / 3.0                  # Richardson in 1/s
        # 0.9984 = 1 - (kh)^2/6 measured for every term; a planted coefficient error moves one >= 12%
        assert c == pytest.approx(1.0 - (K / N) ** 2 / 6.0, abs=0.005), (key, TERMS[key[1]], c)
