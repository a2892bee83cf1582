"""Host logic of bench.py on the CPU: the algorithmic bytes the roofline
divides by, the tile size it charges live cells by, and the clock record
taken from nvidia-smi samples (which decides whether a run is kept)."""
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _w(dim, n_cells, weighted=False):
    return types.SimpleNamespace(dim=dim, n_cells=n_cells, knots=[0.0, 1.0] if weighted else None, bunch=None)


def test_algorithmic_bytes_per_unit():
    # 3D, constant weight: 28 B of state per particle (packed cell 4, three
    # offsets 12, momentum 12), read and written in a live tile; 16 B per
    # streamed slot (cell and momentum read); 36 B per live cell (E, B read
    # for the gather, J written); 60 B per cell for the field update
    w = _w(3, 1000)
    step, push, sp = bench.algorithmic_bytes(w, 10_000, streamed=6_000, live_cells=200)
    assert sp == 28
    assert push == 4_000 * 56 + 6_000 * 16 + 200 * 36
    assert step == push + 1000 * 60
    # every cell live by default; a live-cell count above the grid is capped
    assert bench.algorithmic_bytes(w, 10, 0)[1] == 10 * 56 + 1000 * 36
    assert bench.algorithmic_bytes(w, 10, 0, live_cells=5000)[1] == 10 * 56 + 1000 * 36
    # 2D with per-particle weights: 4 + 8 + 12 + 4 = 28 B as well; 3D with weights 32 B
    assert bench.algorithmic_bytes(_w(2, 64, weighted=True), 1)[2] == 28
    assert bench.algorithmic_bytes(_w(3, 64, weighted=True), 1)[2] == 32


def test_tile_cells():
    assert bench.tile_cells(_w(3, 1), None) == 512
    assert bench.tile_cells(_w(2, 1), {}) == 256
    assert bench.tile_cells(_w(3, 1), {"tile": [8, 8, 4]}) == 256
    assert bench.tile_cells(_w(2, 1), {"tile": [32, 32, 1]}) == 1024


def _line(sm, mx, active=(), power=900.0):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ["Active" if nm in active else "Not Active" for nm in names]
    return ", ".join(["0", str(sm), str(mx), str(power), "0x0"] + flags)


def test_clock_record():
    text = "\n".join([_line(2070, 2070), _line(1980, 2070, ("sw_power_cap",)), _line(2070, 2070),
                      "garbage line", _line("[N/A]", 2070)])
    rec = bench.parse_clocks(text)
    assert rec["samples"] == 3
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]
    rec = bench.parse_clocks(_line(1400, 2070, ("hw_slowdown", "hw_thermal_slowdown")))
    assert rec["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"] and rec["sm_mhz"] == 1400.0
    assert bench.parse_clocks("") is None
    assert bench.parse_clocks("a, b") is None


if __name__ == "__main__":
    sys.exit(pytest.main([__file__, "-q"]))
