"""Pins for the oracle's full timestep (Sec. 2 loop; Sec. 2 moving window).

* Cold plasma, k = 0 mode: every electron starts with the same small u_x in a
  neutral periodic box.  The loop then reduces to the leapfrog oscillator
  E^{n+1} - 2 E^n + E^{n-1} = -omega_p^2 dt^2 E^n, i.e. the discrete relation
  sin(omega dt / 2) = omega_p dt / 2, whatever the shape order.
* Charge conservation of the whole loop: div E^n - (rho^n - rho^0) stays at
  round-off relative to rho (thermal plasma, every order, 2D and 3D).
* Moving window: a windowed run equals a fixed larger box, seen in the
  window frame, away from the rear boundary.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1310_0930_gb300 import inputs


def _load(sim, w: inputs.Workload, parts: inputs.Particles):
    x = np.zeros((3, parts.n))
    x[: w.dim] = parts.positions64()
    sim.load(x, parts.u.astype(np.float64), parts.w.astype(np.float64),
             capacity=int(parts.n * 1.2) + 64)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_cold_plasma_k0_oscillation_discrete_frequency(p):
    dt = 0.5  # omega_p dt = 0.5; Courant number 0.71 on d = 1 cells
    w = inputs.Workload("cold", 2, (8, 8), (1.0, 1.0), dt, p, (2, 2), 1.0)
    parts = inputs.background(w)
    parts.u[0] = 1e-4
    sim = oracle.Sim(2, w.n, w.d, dt, p)
    _load(sim, w, parts)
    ex = []
    for _ in range(60):
        sim.step(1)
        exf = sim.field("Ex")
        assert np.ptp(exf) < 1e-8 * 1e-4  # stays uniform (round-off only, relative to u0)
        ex.append(exf.mean())
    ex = np.array(ex)
    amp = np.max(np.abs(ex))
    c = 1 - dt * dt / 2  # cos(omega dt) with omega_p = 1
    resid = ex[2:] - 2 * c * ex[1:-1] + ex[:-2]
    assert np.max(np.abs(resid)) < 1e-7 * amp
    # and the amplitude is the one set by the initial current: E ~ u0 / omega_p
    assert 0.9e-4 < amp < 1.1e-4


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3)])
def test_gauss_law_residual_at_roundoff(dim, p):
    if dim == 2:
        w = inputs.thermal_2d(n=(16, 12), steps=15, order=p)
        w.uth = 0.08
    else:
        w = inputs.thermal_3d(n=(8, 6, 7), steps=6, order=p)
    parts = inputs.background(w)
    sim = oracle.Sim(dim, w.n, w.d, w.dt, p)
    _load(sim, w, parts)
    rho0 = sim.charge()
    for _ in range(w.steps):
        sim.step(1)
        r = sim.div_e() - (sim.charge() - rho0)
        assert np.max(np.abs(r)) < 1e-12 * np.max(np.abs(rho0))
    assert np.max(np.abs(sim.E)) > 1e-4  # fields did develop


def test_moving_window_equals_fixed_box_in_window_frame():
    """Vacuum laser followed by a window vs. the same laser in a longer fixed
    box, plus a cold plasma slab the window injects as it moves."""
    base = dict(dim=2, d=(1.0, 0.3), dt=0.27, order=2)
    laser = dict(a0=0.3, waist=12.0, fwhm=6.0, plane=4)
    nwin, nbig, nx = 200, 300, 48
    t0 = 40.0     # pulse peak then sits ~97 cells into the window
    steps = 220
    win = inputs.Workload("w", 2, (nx, nwin), (1.0, 0.3), 0.27, 2, (2, 2), 0.01, open_last=True)
    big = inputs.Workload("b", 2, (nx, nbig), (1.0, 0.3), 0.27, 2, (2, 2), 0.01, open_last=True)
    sw = oracle.Sim(2, (nx, nwin), base["d"], base["dt"], 2, open_last=True, laser=laser,
                    window=dict(v=1.0, t0=t0, ppc=(2, 2), density=0.01))
    sb = oracle.Sim(2, (nx, nbig), base["d"], base["dt"], 2, open_last=True, laser=laser)
    _load(sw, win, inputs.background(win))
    _load(sb, big, inputs.background(big))
    sw.step(steps)
    sb.step(steps)
    S = sw.shifts
    assert S > 50
    exw = sw.field("Ex")
    exb = sb.field("Ex")
    # compare the front 70% of the window (rear boundary effects stay at the rear)
    lo = int(0.3 * nwin)
    a = exw[lo:nwin - 1]
    b = exb[lo + S:nwin - 1 + S]
    assert np.max(np.abs(a)) > 0.2
    np.testing.assert_allclose(a, b, atol=1e-6 * 0.3)
    # particles: same count of electrons inside the compared region
    xw, _, _ = sw.particles()
    xb, _, _ = sb.particles()
    cw = np.sum((xw[1] >= lo) & (xw[1] < nwin - 4))
    cb = np.sum((xb[1] >= lo + S) & (xb[1] < nwin - 4 + S))
    assert cw == cb
