"""Pins for the oracle's energy diagnostics and the density profile of the
plasma a moving window injects (Sec. 2: the loop's energy bookkeeping and the
laser-wakefield setup).

* Kinetic energy W_kin = V sum w m (gamma - 1): particles with negligible
  weight in a uniform electric field of a periodic box gain exactly
  q E dt / m of momentum per step (pure-E Boris), so after K steps
  u = u0 + K q E dt / m in closed form and the relativistic kinetic energy
  of the w V physical particles each macro-particle stands for is known.
  Non-unit cell sizes and mass make a missing cell volume, weight or mass
  factor, or gamma in place of gamma - 1, fail.
* Work-energy theorem along the leapfrog path: the kinetic energy gained in a
  step equals the work q E . dx of the field on the step's displacement to
  second order in the momentum kick.
* Field energy against kinetic energy: in a cold k = 0 plasma oscillation
  the energy moves between W_E = 1/2 sum E^2 V and W_kin; their sum stays
  within the leapfrog bound (the kinetic energy is taken half a step behind
  the field energy), and each reaches the same peak.
* Density profile with knots: every particle a moving window injects carries
  w = n(z_lab) / (particles per cell), n piecewise linear through knots
  equally spaced over [z0, z1] and constant outside; the expected value is
  numpy's own linear interpolation at the particle's lab position.
"""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("dim", [2, 3])
def test_kinetic_energy_of_particles_accelerated_by_a_uniform_field(dim):
    n = (6, 5, 4)[:dim]
    d = (0.3, 0.5, 0.7)[:dim]
    dt = 0.1
    q, m = -1.0, 1.7
    E0 = np.array([0.02, -0.03, 0.01])
    sim = oracle.Sim(dim, n, d, dt, 2, q=q, m=m, nthreads=1)
    for c, name in enumerate(("Ex", "Ey", "Ez")):
        sim.field(name)[...] = E0[c]
    x = np.zeros((3, 3))
    x[:dim] = np.array([[1.2, 3.7, 4.05], [0.4, 2.5, 4.9], [0.3, 1.1, 3.6]])[:dim]
    u0 = np.array([[0.0, 0.1, -0.4], [0.0, 0.0, 0.3], [0.0, 0.2, 0.0]])
    w = np.array([1e-12, 2e-12, 3e-12])  # self-fields ~1e-12 of E0
    sim.load(x, u0, w)
    K = 60
    sim.step(K)
    _, u, _ = sim.particles()
    u_exact = u0 + K * q * dt / m * E0[:, None]
    np.testing.assert_allclose(u, u_exact, rtol=0, atol=1e-12)
    V = float(np.prod(d))
    gamma = np.sqrt(1.0 + np.sum(u_exact ** 2, axis=0))
    w_kin = V * np.sum(w * m * (gamma - 1.0))
    got = sim.energies()["W_kin"]
    assert abs(got - w_kin) <= 1e-9 * w_kin, (got, w_kin)
    # the field energy of the uniform field: 1/2 |E|^2 times the box volume
    w_e = 0.5 * float(np.sum(E0 ** 2)) * V * int(np.prod(n))
    assert abs(sim.energies()["W_E"] - w_e) <= 1e-9 * w_e


def test_work_energy_theorem_along_the_leapfrog_path():
    n, d, dt = (8, 8, 8), (0.4, 0.4, 0.4), 0.05
    q, m = -1.0, 1.0
    E0 = np.array([0.3, 0.0, -0.2])
    sim = oracle.Sim(3, n, d, dt, 1, q=q, m=m, nthreads=1)
    for c, name in enumerate(("Ex", "Ey", "Ez")):
        sim.field(name)[...] = E0[c]
    x = np.array([[2.5], [3.5], [4.5]])
    sim.load(x, np.array([[0.5], [0.0], [0.2]]), np.array([1e-12]))
    V = float(np.prod(d))
    du = abs(q) * dt / m * float(np.linalg.norm(E0))  # momentum kick per step
    for _ in range(40):
        k0 = sim.energies()["W_kin"]
        x0 = sim.particles()[0].copy()
        sim.step(1)
        k1 = sim.energies()["W_kin"]
        dx = (sim.particles()[0] - x0)[:, 0] * np.array(d)  # displacement (no wrap in 40 steps here)
        work = q * float(E0 @ dx) * 1e-12 * V  # on the w V physical particles
        assert abs((k1 - k0) - work) <= 1e-12 * V * du * du, (k1 - k0, work)


def test_field_and_kinetic_energy_exchange_in_a_cold_oscillation():
    d, dt = (0.5, 0.25), 0.1  # omega_p dt = 0.1; Courant number 0.45
    n = (8, 8)
    sim = oracle.Sim(2, n, d, dt, 2, nthreads=1)
    ppc = 4
    xs = []
    for j in range(n[1]):
        for i in range(n[0]):
            for a in range(2):
                for b in range(2):
                    xs.append((i + 0.25 + 0.5 * a, j + 0.25 + 0.5 * b))
    x = np.zeros((3, len(xs)))
    x[:2] = np.array(xs).T
    u = np.zeros((3, len(xs)))
    u[0] = 1e-3
    sim.load(x, u, np.full(len(xs), 1.0 / ppc))  # density 1: omega_p = 1
    tot, we, wk = [], [], []
    for _ in range(140):  # about two plasma periods
        sim.step(1)
        e = sim.energies()
        we.append(e["W_E"])
        wk.append(e["W_kin"])
        tot.append(e["W_E"] + e["W_B"] + e["W_kin"])
    tot = np.array(tot)
    assert (tot.max() - tot.min()) <= 0.1 * tot.mean()
    assert abs(max(we) - max(wk)) <= 0.05 * max(wk)
    # and the scale: kinetic energy of the initial drift, n m u0^2 / 2 over the box
    box = float(np.prod(n)) * float(np.prod(d))
    assert abs(max(wk) - 0.5 * 1e-6 * box) <= 0.05 * 0.5 * 1e-6 * box


def test_injected_plasma_follows_the_piecewise_linear_profile():
    dim, n, d, dt = 2, (8, 64), (1.0, 0.3), 0.27
    ppc = (2, 3)
    knots = np.array([0.002, 0.004, 0.001, 0.003, 0.003, 0.0005])
    z0, z1 = 31.0, 41.0  # the profile spans part of the injected plasma the window still holds
    sim = oracle.Sim(dim, n, d, dt, 2, open_last=True, nthreads=1,
                     window=dict(v=1.0, t0=0.0, ppc=ppc, density=0.0, knots=knots, z0=z0, z1=z1))
    sim.load(np.zeros((3, 0)), np.zeros((3, 0)), np.zeros(0), capacity=40000)
    sim.step(100)  # 91 shifts: the window holds plasma injected at lab z from 28 to 45
    S = sim.shifts
    assert S > 80
    x, u, w = sim.particles()
    assert len(w) > 1000 and not np.any(u)  # cold, and no fields to move them
    zlab = (x[1] + S) * d[1]
    kz = np.linspace(z0, z1, len(knots))
    expect = np.interp(zlab, kz, knots) / (ppc[0] * ppc[1])
    np.testing.assert_allclose(w, expect, rtol=1e-12, atol=0)
    # the injected layers cover the profile's whole range, both clamped ends included
    assert zlab.min() < z0 and zlab.max() > z1
