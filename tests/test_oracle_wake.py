"""Pin for the oracle's laser-plasma coupling (Sec. 2 LWFA runs): the linear
wakefield of a weak Gaussian pulse.

A plane, linearly polarised pulse a(xi) = a0 exp(-xi^2/L^2) cos(xi) (xi = z - t,
units c = omega0 = 1, density n in units of n_c, so k_p^2 = n) in a cold
underdense plasma drives, to first order in a0^2, a potential with
(d^2/dxi^2 + k_p^2) phi = k_p^2 <a^2>/2 and <a^2> = (a0^2/2) exp(-2 xi^2/L^2).
Behind the pulse phi oscillates with amplitude (k_p/2) |int <a^2> e^{i k_p xi} dxi|,
so the longitudinal field E = -dphi/dxi peaks at

    E_max = k_p^2 a0^2 L sqrt(pi/2) exp(-k_p^2 L^2 / 8) / 4,

quadratic in a0, and the wake has the pulse's group velocity sqrt(1 - n), i.e.
the wavelength 2 pi sqrt(1 - n) / k_p.  The antenna's envelope is Gaussian in
intensity with FWHM tau, so L = tau / sqrt(2 ln 2).  A transversely uniform
pulse (waist far wider than the periodic box) makes the 2D run one-dimensional;
the plasma is loaded cold and regular.  The oracle agrees with the amplitude to
a few per cent (the remaining terms are of order a0^2, n and the grid
dispersion) and with the wavelength to well under one per cent.
"""
import math

import numpy as np

import oracle
from paper_1310_0930_gb300 import inputs

NZ, DENS, TAU, T = 900, 0.01, 24.0, 240.0


def _wake(a0):
    w = inputs.Workload("wake", 2, (16, NZ), (1.0, 0.3), 0.27, 2, (1, 4), DENS, open_last=True)
    parts = inputs.background(w)
    sim = oracle.Sim(2, w.n, w.d, w.dt, 2, open_last=True,
                     laser=dict(a0=a0, waist=1e4, fwhm=TAU, plane=4))
    x = np.zeros((3, parts.n))
    x[:2] = parts.positions64()
    sim.load(x, parts.u.astype(np.float64), parts.w.astype(np.float64), capacity=parts.n + 64)
    sim.step(int(round(T / w.dt)))
    z = np.arange(NZ) * w.d[1]
    ez = sim.field("Ey").mean(axis=1)  # the propagation axis is the last one (component 1 in 2D)
    z_pulse = z[np.argmax(np.abs(sim.field("Ex")).max(axis=1))]
    return z, ez, z_pulse


def test_linear_wake_amplitude_wavelength_and_a0_squared_scaling():
    kp = math.sqrt(DENS)
    L = TAU / math.sqrt(2 * math.log(2))
    theory = {}
    measured = {}
    for a0 in (0.1, 0.2):
        z, ez, z_pulse = _wake(a0)
        behind = (z > 10.0) & (z < z_pulse - 2 * L)
        measured[a0] = np.max(np.abs(ez[behind]))
        theory[a0] = kp * kp * a0 * a0 * L * math.sqrt(math.pi / 2) * math.exp(-kp * kp * L * L / 8) / 4
        assert abs(measured[a0] / theory[a0] - 1) < 0.06, (a0, measured[a0], theory[a0])
        # wavelength from the zero crossings behind the pulse (half a wavelength apart)
        zb, eb = z[behind], ez[behind]
        cross = zb[1:][np.sign(eb[1:]) != np.sign(eb[:-1])]
        assert len(cross) >= 4
        lam = 2 * np.mean(np.diff(cross))
        lam_theory = 2 * math.pi * math.sqrt(1 - DENS) / kp
        assert abs(lam / lam_theory - 1) < 0.01, (lam, lam_theory)
    # ponderomotive drive: quadratic in a0
    assert abs(measured[0.2] / measured[0.1] / 4 - 1) < 0.02
