"""3D field-tile staging by the tensor-memory accelerator (tuning tma = 1):
on a grid with interior tiles (whose field box lies inside the stored grid)
it gives the fields of the default plain staging and of the oracle, and no
bounded wait on the tile barrier gives up."""
import pytest

from gpu_helpers import FIELD_NAMES, pair, rel_l2
from paper_1310_0930_gb300 import inputs
from paper_1310_0930_gb300.sim import Simulation

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("order", [1, 2, 3])
def test_tma_staging_matches_plain_and_oracle(order):
    # 8x8x8 tiles: those at origins 8..16 (x, y) and 8..32 (z) are interior
    w = inputs.thermal_3d(n=(32, 32, 48), steps=12, order=order)
    parts = inputs.background(w)
    gpu, orc = pair(w, parts, tuning={"tma": 1})
    plain = Simulation(w)
    plain.load(parts)
    gpu.step(w.steps)
    plain.step(w.steps)
    orc.step(w.steps)
    dg, dp = gpu.diagnostics(), plain.diagnostics()
    assert dg["status"] == 0 and dp["status"] == 0
    for name in FIELD_NAMES:
        ref = orc.field(name)
        assert rel_l2(gpu.field(name), plain.field(name)) <= 1e-6, name
        assert rel_l2(gpu.field(name), ref) <= 1e-4, name
    gpu.close()
    plain.close()
