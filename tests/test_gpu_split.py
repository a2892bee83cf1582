"""The virtual-trajectory deposit (pic_tuning.deposit = 1; Sec. 5.2 step iv)
against the oracle's split deposit: one step with every particle's current
compared (through J), and a hundred steps of fields and the device's Gauss
residual; the split current differs from the undivided one, so the variant
is the one that ran.

Tolerances as in the other parity tests: J and fields after one step
relative L2 <= 1e-5, fields after 100 steps <= 1e-4, Gauss residual <= 1e-6.
"""
import numpy as np
import pytest

from gpu_helpers import FIELD_NAMES, pair, rel_l2, smooth_fields
from paper_1310_0930_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,order", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2), (3, 3)])
def test_split_one_step_current_matches_oracle(dim, order):
    if dim == 2:
        w = inputs.thermal_2d(n=(48, 32), order=order)
    else:
        w = inputs.thermal_3d(n=(16, 16, 24), order=order)
    w.uth = 0.3  # fast enough that many moves cross node boundaries
    parts = inputs.background(w)
    fields = smooth_fields(w, amp=0.05)
    gpu, orc = pair(w, parts, fields=fields, tuning={"deposit": 1})
    ref, _ = pair(w, parts, fields=fields)  # undivided deposit, same state
    gpu.step(1)
    orc.step(1)
    ref.step(1)
    for name in ("Jx", "Jy", "Jz"):
        a = gpu.field(name)
        assert rel_l2(a, orc.field(name)) <= 1e-5, name
    # the split current is not the undivided one
    diff = max(rel_l2(gpu.field(n), ref.field(n)) for n in ("Jx", "Jy"))
    assert diff > 1e-4, diff
    gpu.close()
    ref.close()


@pytest.mark.parametrize("dim,order", [(2, 2), (3, 2)])
def test_split_100_steps_fields_and_gauss(dim, order):
    if dim == 2:
        w = inputs.thermal_2d(steps=100, order=order)
        w.uth = 0.05
    else:
        w = inputs.thermal_3d(n=(16, 16, 16), steps=40, order=order)
        w.uth = 0.05
    parts = inputs.background(w)
    gpu, orc = pair(w, parts, tuning={"deposit": 1})
    gpu.step(w.steps)
    orc.step(w.steps)
    for name in FIELD_NAMES:
        assert rel_l2(gpu.field(name), orc.field(name)) <= 1e-4, name
    assert gpu.diagnostics()["gauss_resid"] <= 1e-6
    gpu.close()
