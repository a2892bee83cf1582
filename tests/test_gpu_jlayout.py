"""The four-component current layout (pic_tuning.j_layout = 1; Sec. 5.1:
x, y, z and an unused lane per node, the tile current added by one 16-byte
vector atomic per node) against the oracle and against the three-array
layout: one step of current, 100 steps of a thermal plasma, and a 3D LWFA
with laser, zero-field tiles, Mur ends and a moving window.

Tolerances as in the other parity tests."""
import numpy as np
import pytest

from gpu_helpers import FIELD_NAMES, pair, rel_l2, smooth_fields
from paper_1310_0930_gb300 import inputs
from paper_1310_0930_gb300.sim import Simulation

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,order", [(2, 2), (3, 1), (3, 2)])
def test_four_component_current_one_step(dim, order):
    if dim == 2:
        w = inputs.thermal_2d(n=(48, 32), order=order)
    else:
        w = inputs.thermal_3d(n=(16, 16, 24), order=order)
    w.uth = 0.2
    parts = inputs.background(w)
    fields = smooth_fields(w, amp=0.05)
    gpu, orc = pair(w, parts, fields=fields, tuning={"j_layout": 1})
    gpu.step(1)
    orc.step(1)
    for name in ("Jx", "Jy", "Jz") + tuple(FIELD_NAMES):
        assert rel_l2(gpu.field(name), orc.field(name)) <= 1e-5, name
    gpu.close()


def test_four_component_current_100_steps_2d():
    w = inputs.thermal_2d(steps=100)
    w.uth = 0.05
    parts = inputs.background(w)
    gpu, orc = pair(w, parts, tuning={"j_layout": 1})
    gpu.step(w.steps)
    orc.step(w.steps)
    for name in FIELD_NAMES:
        assert rel_l2(gpu.field(name), orc.field(name)) <= 1e-4, name
    assert gpu.diagnostics()["gauss_resid"] <= 1e-6
    gpu.close()


def test_four_component_current_lwfa_3d_equals_three_arrays():
    w = inputs.lwfa_3d(n=(16, 16, 96), steps=50)
    w.laser.a0, w.laser.waist, w.laser.fwhm = 1.5, 5.0, 6.0
    w.window.t0 = 8.0
    parts = inputs.background(w)
    a = Simulation(w, tuning={"j_layout": 1})
    b = Simulation(w)
    a.load(parts)
    b.load(parts)
    a.step(w.steps)
    b.step(w.steps)
    da, db = a.diagnostics(), b.diagnostics()
    assert da["shifts"] == db["shifts"] > 5 and da["n_particles"] == db["n_particles"]
    assert da["status"] == 0
    for name in tuple(FIELD_NAMES) + ("Jx", "Jy", "Jz"):
        assert rel_l2(a.field(name), b.field(name)) <= 1e-5, name
    a.close()
    b.close()
