"""Edge cases of the CUDA path: particles on cell faces and just below the
next face with relativistic momenta in smooth random fields (against the
oracle, particle by particle), fields confined to part of the grid (tiles
whose staged fields are all zero take the zero-force path), cold plasma in
zero fields (bit-identical after stepping), a run whose tiles are mostly
empty (a single particle per tile at most), and a load beyond the configured
capacity (refused with PIC_EOVERFLOW, nothing written)."""
import numpy as np
import pytest

from gpu_helpers import FIELD_NAMES, pair, rel_l2, smooth_fields
from paper_1310_0930_gb300 import abi, inputs
from paper_1310_0930_gb300.sim import Simulation

pytestmark = pytest.mark.gpu


def _compare_particles(gpu, orc, n, dims, tol_u=1e-5, tol_x=4e-6):
    g = gpu.particles()
    assert g["n"] == n
    order = np.argsort(g["id"])
    assert np.array_equal(g["id"][order], np.arange(n))
    xo, uo, _ = orc.particles()
    ug = g["u"][:, order].astype(np.float64)
    du = np.linalg.norm(ug - uo, axis=0) / np.maximum(np.linalg.norm(uo, axis=0), 1e-7)
    assert np.max(du) < tol_u, np.max(du)
    xg = g["cell"][:, order].astype(np.float64) + g["off"][:, order]
    dx = xg - xo[: len(dims)]
    dx -= np.round(dx / np.array(dims)[:, None]) * np.array(dims)[:, None]
    assert np.max(np.abs(dx)) < tol_x, np.max(np.abs(dx))


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_face_offsets_and_relativistic_momenta_3d(order):
    """Offsets 0 and the largest float below 1 on every axis, |u| up to 50
    (gamma ~ 50, moves close to the Courant limit), 4 steps in smooth fields."""
    w = inputs.thermal_3d(n=(16, 16, 24), steps=4, order=order)
    rng = np.random.default_rng(5)
    n = 2000
    cell = np.stack([rng.integers(0, m, n) for m in w.n]).astype(np.int32)
    below1 = np.nextafter(np.float32(1.0), np.float32(0.0))
    off = rng.choice(np.array([0.0, below1, 0.5, 0.25], np.float32), size=(3, n))
    u = (rng.normal(size=(3, n)) * rng.choice([0.01, 1.0, 30.0], size=n)).astype(np.float32)
    wgt = np.full(n, 0.1, np.float32)
    parts = inputs.Particles(cell, off.astype(np.float32), u, wgt)
    fields = smooth_fields(w, amp=0.2)
    gpu, orc = pair(w, parts, fields=fields, per_particle_weight=True)
    gpu.step(w.steps)
    orc.step(w.steps)
    _compare_particles(gpu, orc, n, w.n)
    for name in FIELD_NAMES:  # (the imposed fields are not Gauss-consistent: no residual check)
        assert rel_l2(gpu.field(name), orc.field(name)) < 1e-5, name
    gpu.close()


def test_sparse_particles_mostly_empty_tiles_2d():
    """64x48 cells, 16x16 tiles, 7 particles: most tiles hold none."""
    w = inputs.thermal_2d(n=(64, 48), steps=20)
    rng = np.random.default_rng(9)
    n = 7
    cell = np.stack([rng.integers(0, m, n) for m in w.n]).astype(np.int32)
    off = rng.uniform(0, 1, size=(2, n)).astype(np.float32)
    u = rng.normal(0, 0.3, size=(3, n)).astype(np.float32)
    parts = inputs.Particles(cell, off, u, np.full(n, 1.0, np.float32))
    gpu, orc = pair(w, parts, per_particle_weight=True)
    gpu.step(w.steps)
    orc.step(w.steps)
    _compare_particles(gpu, orc, n, w.n)
    for name in FIELD_NAMES:
        assert rel_l2(gpu.field(name), orc.field(name)) < 1e-5, name
    gpu.close()


def test_load_beyond_capacity_is_refused():
    """With a configured capacity, a load that would leave no room for the
    moving window's injected layers is refused with PIC_EOVERFLOW and writes
    nothing: the particles already loaded are intact and step on."""
    w = inputs.lwfa_2d(nx=32, nz=64, steps=10)
    parts = inputs.background(w)
    half = parts.n // 2
    first, second = parts.subset(np.arange(half)), parts.subset(np.arange(half, parts.n))
    # (fixed sort interval 4: the injection room is (4 + 2) shifts of particles)
    sim = Simulation(w, capacity=half + 12 * 32 * 4 + 4096, tuning={"sort_interval": 4, "sort_policy": 1})
    sim.load(first)
    with pytest.raises(abi.PicError) as err:
        sim.load(second)
    assert err.value.code == abi.PIC_EOVERFLOW
    sim.step(w.steps)
    d = sim.diagnostics()
    assert d["status"] == 0 and d["n_particles"] == half
    sim.close()


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_fields_in_part_of_the_grid_3d(order):
    """Smooth fields in the lower half of z only, exact zeros elsewhere; moving
    particles everywhere.  Tiles whose staged fields are all zero take the
    zero-force path (no gather), the others the full gather; both against the
    oracle, particle by particle, over 3 steps."""
    w = inputs.thermal_3d(n=(16, 16, 48), steps=3, order=order)
    rng = np.random.default_rng(11)
    n = 6000
    cell = np.stack([rng.integers(0, m, n) for m in w.n]).astype(np.int32)
    off = rng.uniform(0, 1, size=(3, n)).astype(np.float32)
    u = rng.normal(0, 0.2, size=(3, n)).astype(np.float32)
    parts = inputs.Particles(cell, off, u, np.full(n, 0.05, np.float32))
    fields = smooth_fields(w, amp=0.2)
    for name in FIELD_NAMES:  # (arrays are [z][y][x])
        fields[name][w.n[2] // 2:] = 0.0
    gpu, orc = pair(w, parts, fields=fields, per_particle_weight=True)
    gpu.step(w.steps)
    orc.step(w.steps)
    _compare_particles(gpu, orc, n, w.n)
    for name in FIELD_NAMES:
        assert rel_l2(gpu.field(name), orc.field(name)) < 1e-5, name
    gpu.close()


def test_cold_plasma_in_zero_fields_is_unchanged():
    """Particles at rest with E = B = 0 everywhere: after 5 steps every cell,
    offset and momentum is bit-identical to the load and J and the fields are
    exactly zero (the zero-force path must not change anything)."""
    w = inputs.thermal_3d(n=(16, 16, 32), steps=5, order=2)
    rng = np.random.default_rng(12)
    n = 5000
    cell = np.stack([rng.integers(0, m, n) for m in w.n]).astype(np.int32)
    off = rng.uniform(0, 1, size=(3, n)).astype(np.float32)
    u = np.zeros((3, n), np.float32)
    parts = inputs.Particles(cell, off, u, np.full(n, 0.05, np.float32))
    sim = Simulation(w, track_ids=True, per_particle_weight=True)
    sim.load(parts)
    sim.step(w.steps)
    g = sim.particles()
    order = np.argsort(g["id"])
    assert np.array_equal(g["cell"][:, order], cell)
    assert np.array_equal(g["off"][:, order], off)
    assert np.array_equal(g["u"][:, order], u)
    for name in FIELD_NAMES + ["Jx", "Jy", "Jz"]:
        assert not np.any(sim.field(name)), name
    sim.close()
