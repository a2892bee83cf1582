"""The FP64 oracle reproduces its recorded energy history (a regression pin
written by tests/golden/make_golden.py from the oracle alone); single-thread
oracle runs are deterministic, so the match is to round-off."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden  # noqa: E402


def test_oracle_reproduces_recorded_energy_history():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "thermal_2d_32x32_energies.txt")
    ref = np.loadtxt(path)
    got = np.array(make_golden.thermal_energies(steps=int(ref[-1, 0])))
    assert np.array_equal(got[:, 0], ref[:, 0])
    assert np.allclose(got[:, 1:], ref[:, 1:], rtol=1e-12, atol=0.0)
