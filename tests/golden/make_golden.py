"""Write the regression fixtures of this folder from the FP64 oracle alone
(no GPU code).  Run from the repository root:

    python tests/golden/make_golden.py

thermal_2d_32x32_energies.txt: the oracle's field and kinetic energies of a
seeded 32x32 warm plasma (the 2D thermal configuration on a smaller grid,
quadratic shape), one line per step.  The paper prints no worked example
values for the method, so these fixtures pin the oracle against its own
history; its correctness is pinned by the closed-form tests."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1310_0930_gb300 import inputs  # noqa: E402


def thermal_energies(steps=20):
    w = inputs.thermal_2d(n=(32, 32), steps=steps)
    parts = inputs.background(w)
    sim = oracle.Sim(w.dim, w.n, w.d, w.dt, w.order, nthreads=1)
    x = np.zeros((3, parts.n))
    x[:2] = parts.positions64()
    sim.load(x, parts.u.astype(np.float64), parts.w.astype(np.float64))
    rows = []
    for s in range(steps):
        sim.step(1)
        e = sim.energies()
        rows.append((s + 1, e["W_E"], e["W_B"], e["W_kin"]))
    return rows


def main():
    rows = thermal_energies()
    with open(os.path.join(HERE, "thermal_2d_32x32_energies.txt"), "w") as f:
        f.write("# FP64 oracle, 2D warm plasma 32x32 cells, d=0.2, dt=0.14, 2x2 ppc, u_th=0.01, quadratic, seed 1\n")
        f.write("# written by tests/golden/make_golden.py; columns: step W_E W_B W_kin\n")
        for r in rows:
            f.write("%d %.17e %.17e %.17e\n" % r)


if __name__ == "__main__":
    main()
