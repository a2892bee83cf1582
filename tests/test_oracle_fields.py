"""Pins for the oracle's Yee field solver, its open boundary and the laser
antenna (Sec. 2 FDTD solver; Sec. 2 laser driver).

* Discrete standing waves: for a divergence-free eigenmode of curl^T curl with
  eigenvalue kappa^2 = sum_a (2 sin(k_a d_a / 2) / d_a)^2, the B-half / E / B-half
  update is velocity Verlet, so starting with B = 0 (or E = 0) the mode evolves
  as cos(n Omega dt) exactly, with cos(Omega dt) = 1 - kappa^2 dt^2 / 2, i.e. the
  Yee numerical dispersion relation (sin(Omega dt / 2) / dt)^2 = sum (sin(k d/2)/d)^2.
* div B stays zero and div E stays unchanged in vacuum.
* First-order Mur: a pulse leaving through the open axis is absorbed.
* The antenna launches a one-way pulse with peak a0 and the Gaussian-beam
  energy a0^2 w0 sqrt(pi/2) * fwhm sqrt(pi / (4 ln 2)) / 2 (2D).
"""
import math

import numpy as np
import pytest

import oracle


def _omega(k, d, dt):
    kap2 = sum((2 * math.sin(ka * da / 2) / da) ** 2 for ka, da in zip(k, d))
    return math.acos(1 - kap2 * dt * dt / 2) / dt


def _grid(sim):
    s = sim.s
    if s.dim == 3:
        k, j, i = np.meshgrid(np.arange(s.n[2]), np.arange(s.n[1]), np.arange(s.n[0]), indexing="ij")
        return i, j, k
    j, i = np.meshgrid(np.arange(s.n[1]), np.arange(s.n[0]), indexing="ij")
    return i, j, None


def test_yee_2d_tm_standing_wave_follows_discrete_dispersion():
    n, d, dt = (24, 16), (0.3, 0.5), 0.2
    sim = oracle.Sim(2, n, d, dt, 2)
    i, j, _ = _grid(sim)
    k = (2 * math.pi * 3 / (n[0] * d[0]), 2 * math.pi * 2 / (n[1] * d[1]))
    ez0 = np.cos(k[0] * i * d[0] + k[1] * j * d[1])
    sim.field("Ez")[:] = ez0
    N = 137
    sim.step(N)
    W = _omega(k, d, dt)
    np.testing.assert_allclose(sim.field("Ez"), math.cos(N * W * dt) * ez0, atol=1e-11)
    # a continuum-dispersion frequency would be visibly off
    wc = math.hypot(*k)
    assert abs(math.cos(N * wc * dt) - math.cos(N * W * dt)) > 1e-2


def test_yee_2d_te_standing_wave_bz():
    n, d, dt = (20, 18), (0.4, 0.3), 0.2
    sim = oracle.Sim(2, n, d, dt, 2)
    i, j, _ = _grid(sim)
    k = (2 * math.pi * 2 / (n[0] * d[0]), 2 * math.pi * 5 / (n[1] * d[1]))
    bz0 = np.cos(k[0] * (i + 0.5) * d[0] + k[1] * (j + 0.5) * d[1])
    sim.field("Bz")[:] = bz0
    N = 91
    sim.step(N)
    W = _omega(k, d, dt)
    np.testing.assert_allclose(sim.field("Bz"), math.cos(N * W * dt) * bz0, atol=1e-11)


def test_yee_3d_standing_waves():
    n, d, dt = (12, 10, 14), (0.5, 0.4, 0.3), 0.15
    sim = oracle.Sim(3, n, d, dt, 2)
    i, j, kk = _grid(sim)
    kE = (2 * math.pi * 2 / (n[0] * d[0]), 0.0, 2 * math.pi * 3 / (n[2] * d[2]))
    kB = (0.0, 2 * math.pi * 1 / (n[1] * d[1]), 2 * math.pi * 2 / (n[2] * d[2]))
    ey0 = np.cos(kE[0] * i * d[0] + kE[2] * kk * d[2])           # E_y at (i, j+1/2, k), no y dependence
    sim.field("Ey")[:] = ey0
    N = 57
    sim.step(N)
    np.testing.assert_allclose(sim.field("Ey"), math.cos(N * _omega(kE, d, dt) * dt) * ey0, atol=1e-11)
    sim2 = oracle.Sim(3, n, d, dt, 2)
    bx0 = np.cos(kB[1] * (j + 0.5) * d[1] + kB[2] * (kk + 0.5) * d[2])  # B_x at (i, j+1/2, k+1/2)
    sim2.field("Bx")[:] = bx0
    sim2.step(N)
    np.testing.assert_allclose(sim2.field("Bx"), math.cos(N * _omega(kB, d, dt) * dt) * bx0, atol=1e-11)


def _div_b(sim):
    s = sim.s
    out = 0
    for a, name in enumerate("xyz"[: s.dim]):
        F = sim.field("B" + name)
        axis = s.dim - 1 - a
        out = out + (np.roll(F, -1, axis=axis) - F) / s.d[a]
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_yee_keeps_div_b_zero_and_div_e_in_vacuum(dim):
    n = (10, 9, 8)[:dim]
    d = (0.3, 0.4, 0.5)[:dim]
    sim = oracle.Sim(dim, n, d, 0.12, 2)
    rng = np.random.default_rng(dim)
    sim.E[:] = rng.normal(size=sim.E.size)
    div0 = sim.div_e()
    sim.step(40)
    assert np.max(np.abs(_div_b(sim))) < 1e-11
    np.testing.assert_allclose(sim.div_e(), div0, atol=1e-11)
    assert np.max(np.abs(sim.B)) > 0.1


def test_mur_absorbs_outgoing_pulse():
    """A plane pulse E_x, B_z = -E_x travelling along +y leaves through the
    open last axis; first-order Mur at normal incidence absorbs it."""
    n, d, dt = (8, 300), (1.0, 0.3), 0.25
    sim = oracle.Sim(2, n, d, dt, 2, open_last=True)
    i, j, _ = _grid(sim)
    y0, width = 200 * d[1], 6.0
    sim.field("Ex")[:] = np.exp(-((j * d[1] - y0) / width) ** 2)
    sim.field("Bz")[:] = -np.exp(-(((j + 0.5) * d[1] - y0) / width) ** 2)
    W0 = sum(sim.energies()[k] for k in ("W_E", "W_B"))
    sim.step(int(50 / dt))  # the pulse crosses the remaining ~30 and leaves
    W1 = sum(sim.energies()[k] for k in ("W_E", "W_B"))
    assert W1 < 1e-3 * W0
    # the reverse direction through the low boundary as well
    sim2 = oracle.Sim(2, n, d, dt, 2, open_last=True)
    sim2.field("Ex")[:] = np.exp(-((j * d[1] - 100 * d[1]) / width) ** 2)
    sim2.field("Bz")[:] = np.exp(-(((j + 0.5) * d[1] - 100 * d[1]) / width) ** 2)
    W0 = sum(sim2.energies()[k] for k in ("W_E", "W_B"))
    sim2.step(int(50 / dt))
    assert sum(sim2.energies()[k] for k in ("W_E", "W_B")) < 1e-3 * W0


def test_laser_antenna_one_way_amplitude_and_energy():
    a0, w0, tau = 0.5, 16.0, 10.0
    n, d, dt = (96, 420), (1.0, 0.3), 0.27
    laser = dict(a0=a0, waist=w0, fwhm=tau, plane=4)
    sim = oracle.Sim(2, n, d, dt, 2, open_last=True, laser=laser)
    steps = int(round(4 * tau / dt))
    sim.step(steps)
    ex = sim.field("Ex")
    peak = np.max(np.abs(ex))
    assert 0.95 * a0 < peak < 1.02 * a0
    # nothing goes backwards: the scattered side of the plane stays dark
    assert np.max(np.abs(ex[:3, :])) < 1e-2 * a0
    W = sum(sim.energies()[k] for k in ("W_E", "W_B"))
    expect = a0 ** 2 * w0 * math.sqrt(math.pi / 2) * tau * math.sqrt(math.pi / (4 * math.log(2))) / 2
    assert abs(W / expect - 1) < 0.03
    # the envelope peak travels at ~c: the peak sits near z = plane + (t - t_peak)
    prof = np.max(np.abs(ex), axis=1)
    zpk = (np.argmax(prof) - 4) * d[1]
    assert abs(zpk - (sim.time - 2 * tau)) < 2.0
