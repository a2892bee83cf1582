"""Zero-field tiles: each step the device classifies the tiles, and those whose
staged field region is all +0 (E = B = 0 at every particle) are advanced by a
streaming kernel instead of the staged tile kernel; quiet tiles (E, B and J
+0 through the step) are left out of the field update.  The results must not
depend on either choice: against the same run with every tile staged
(stream_zero_tiles = 2), with the field update over every tile
(quiet_tiles = 2), and against the FP64 oracle.

Tolerances as in the other parity tests: fields relative L2 <= 1e-5 between
the two device runs (only the order of the FP32 atomic current sums
differs), <= 1e-4 against the oracle; particle and window-shift counts
exact; particles at rest in zero fields bit-identical.
"""
import numpy as np
import pytest

from gpu_helpers import FIELD_NAMES, pair, rel_l2, smooth_fields
from paper_1310_0930_gb300 import inputs
from paper_1310_0930_gb300.sim import Simulation

pytestmark = pytest.mark.gpu


def _by_id(p):
    order = np.argsort(p["id"])
    return {k: (v[..., order] if isinstance(v, np.ndarray) else v) for k, v in p.items()}


def test_lwfa_3d_streamed_tiles_equal_staged_and_oracle():
    # the laser enters through the rear plane: the box ahead of its front is
    # field-free, so most tiles are streamed until the window moves
    w = inputs.lwfa_3d(n=(16, 16, 128), steps=60)
    w.laser.a0, w.laser.waist, w.laser.fwhm = 1.5, 5.0, 6.0
    w.window.t0 = 10.0
    parts = inputs.background(w)
    extra = 16 * 16 * 8 * 40
    # (quiet tiles forced on: at this size the default leaves them off)
    gpu, orc = pair(w, parts, extra=extra, tuning={"quiet_tiles": 1})
    staged = Simulation(w, tuning={"stream_zero_tiles": 2}, track_ids=True)
    staged.load(parts)
    gpu.profile_begin(10)
    gpu.step(10)
    ph, _ = gpu.profile_end()
    assert ph["push_zero"] > 0.0  # the streaming kernel ran
    gpu.step(w.steps - 10)
    staged.step(w.steps)
    orc.step(w.steps)
    d, ds = gpu.diagnostics(), staged.diagnostics()
    assert d["shifts"] == ds["shifts"] == orc.shifts > 5
    assert d["n_particles"] == ds["n_particles"] == orc.np
    assert d["status"] == 0 and ds["status"] == 0
    for name in FIELD_NAMES:
        a = gpu.field(name).astype(np.float64)
        assert rel_l2(a, staged.field(name)) <= 1e-5, name
        assert rel_l2(a, orc.field(name)) <= 1e-4, name
    # every particle by id: the loaded ones (ids below parts.n) and the layers
    # the window injected (numbered after them, the same in both runs)
    pa, pb = _by_id(gpu.particles()), _by_id(staged.particles())
    assert np.array_equal(pa["id"], pb["id"])
    injected = pa["id"] >= parts.n
    assert injected.sum() > 0 and (~injected).sum() > 0 and pa["id"].min() >= 0
    assert np.array_equal(pa["cell"], pb["cell"])
    assert np.max(np.abs(pa["off"] - pb["off"])) <= 1e-5
    assert np.max(np.abs(pa["u"] - pb["u"])) <= 1e-5 * max(1.0, float(np.max(np.abs(pb["u"]))))
    gpu.close()
    staged.close()


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_fields_written_into_a_streamed_region_are_gathered(order):
    """A cold plasma in zero fields is streamed; fields written afterwards
    from the host into half of the box must reach the particles there at the
    next step (writing marks every tile live again)."""
    w = inputs.thermal_3d(n=(32, 16, 16), order=order)
    w.uth = 0.0
    parts = inputs.background(w)
    gpu, orc = pair(w, parts)
    gpu.step(3)
    orc.step(3)
    p0 = _by_id(gpu.particles())
    fields = smooth_fields(w, amp=0.05, seed=5)
    half = np.zeros(tuple(reversed(w.n)), np.float32)
    half[..., : w.n[0] // 2] = 1.0
    for name, arr in fields.items():
        v = (arr * half).astype(np.float32)
        gpu.set_field(name, v)
        orc.field(name)[...] = v.astype(np.float64)
    gpu.step(2)
    orc.step(2)
    p1 = _by_id(gpu.particles())
    moved = np.any(p1["u"] != p0["u"], axis=0)
    assert moved.mean() > 0.3  # the particles in the written half felt the fields
    _, uo, _ = orc.particles()  # (periodic box: the oracle keeps the load order, the ids)
    ou = uo[:, p1["id"]]
    scale = max(float(np.max(np.abs(ou))), 1e-30)
    assert np.max(np.abs(p1["u"] - ou)) <= 1e-5 * scale
    for name in FIELD_NAMES:
        assert rel_l2(gpu.field(name), orc.field(name)) <= 1e-4, name
    gpu.close()


def test_cold_plasma_in_zero_fields_stays_bit_identical_when_streamed():
    w = inputs.lwfa_3d(n=(16, 16, 64), steps=6, with_window=False)
    w.laser = None
    parts = inputs.background(w)
    gpu = Simulation(w, track_ids=True)
    gpu.load(parts)
    p0 = _by_id(gpu.particles())
    gpu.profile_begin(6)
    gpu.step(6)
    ph, _ = gpu.profile_end()
    assert ph["push_zero"] > 0.0
    p1 = _by_id(gpu.particles())
    for k in ("cell", "off", "u"):
        assert np.array_equal(p0[k], p1[k]), k
    for name in FIELD_NAMES + ["Jx", "Jy", "Jz"]:
        assert not np.any(gpu.field(name)), name
    gpu.close()


def test_immobile_plasma_in_imposed_fields_gathers_and_stays():
    """Particles of 1e30 electron masses in smooth imposed fields (the
    frozen-plasma bench in fields): every tile is staged and gathers, no
    particle moves, no current is deposited, and the fields evolve as in
    vacuum, as in the oracle."""
    w = inputs.thermal_3d(n=(16, 16, 24), order=2)
    w.uth = 0.0
    w.mass = 1e30
    parts = inputs.background(w)
    gpu = Simulation(w, track_ids=True)
    gpu.load(parts)
    import oracle
    orc = oracle.Sim(3, w.n, w.d, w.dt, w.order, m=1e30, nthreads=2)
    x = np.zeros((3, parts.n))
    x[:3] = parts.positions64()
    orc.load(x, parts.u.astype(np.float64), parts.w.astype(np.float64))
    for name, arr in smooth_fields(w, amp=0.05, seed=3).items():
        gpu.set_field(name, arr)
        orc.field(name)[...] = arr.astype(np.float64)
    p0 = _by_id(gpu.particles())
    gpu.step(4)
    orc.step(4)
    p1 = _by_id(gpu.particles())
    assert np.array_equal(p0["cell"], p1["cell"]) and np.array_equal(p0["off"], p1["off"])
    assert np.max(np.abs(p1["u"])) < 1e-25
    for name in ("Jx", "Jy", "Jz"):
        assert not np.any(gpu.field(name)), name
    for name in FIELD_NAMES:
        assert rel_l2(gpu.field(name), orc.field(name)) <= 1e-5, name
    gpu.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_quiet_tiles_leave_the_fields_unchanged(dim):
    """The field update over the non-quiet rows of tiles only (quiet_tiles =
    1) against the update over every cell (quiet_tiles = 2), both with the
    zero-field streaming, and against the oracle: a laser entering a plasma
    box through its rear plane and a window that starts moving, so that the
    quiet region ahead of the pulse shrinks, and the window injects plasma
    (slow-path tail particles) at the front."""
    if dim == 3:
        w = inputs.lwfa_3d(n=(16, 16, 128), steps=70)
        w.laser.a0, w.laser.waist, w.laser.fwhm = 1.5, 5.0, 6.0
        w.window.t0 = 10.0
        extra = 16 * 16 * 8 * 60
    else:
        w = inputs.lwfa_2d(nx=32, nz=256, ppc=(2, 2), density=0.01, a0=2.0, waist=8.0, steps=120)
        w.laser.fwhm = 6.0
        w.window.t0 = 18.0
        extra = 32 * 4 * 120
    parts = inputs.background(w)
    on, orc = pair(w, parts, extra=extra, tuning={"quiet_tiles": 1})
    off = Simulation(w, tuning={"quiet_tiles": 2}, track_ids=True)
    off.load(parts)
    on.step(w.steps)
    off.step(w.steps)
    orc.step(w.steps)
    d, do = on.diagnostics(), off.diagnostics()
    assert d["status"] == 0 and do["status"] == 0
    assert d["shifts"] == do["shifts"] == orc.shifts > 5
    assert d["n_particles"] == do["n_particles"] == orc.np
    assert 0 < d["streamed"]
    for name in FIELD_NAMES:
        a = on.field(name).astype(np.float64)
        assert rel_l2(a, off.field(name)) <= 1e-5, name
        assert rel_l2(a, orc.field(name)) <= 1e-4, name
    for name in ("Jx", "Jy", "Jz"):
        assert rel_l2(on.field(name), off.field(name)) <= 1e-5, name
    pa, pb = _by_id(on.particles()), _by_id(off.particles())
    assert np.array_equal(pa["id"], pb["id"]) and np.array_equal(pa["cell"], pb["cell"])
    on.close()
    off.close()
