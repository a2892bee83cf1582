"""The allocation-free charge-density entry point against the regular path.

Some callers cannot allocate device memory: a host framework that hands the
library only buffers it owns, a fixed memory budget, or a loop that must not
allocate once it runs.  pic_charge_density_static serves them from a static
device scratch array.  This test calls it through the C ABI twice in a row on
the same particles (the second call must clear what the first left in the
shared array) and compares both results with pic_read_fields(PIC_RHO) of a
handle holding the same particles and with the FP64 oracle's charge deposit
of the same particles, at the tolerance of the charge checks (FP64
accumulation rounded to FP32: max difference <= 1e-6 of max |rho|).
The file name makes pytest collect it after every other test.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import load_oracle, oracle_for
from paper_1310_0930_gb300 import inputs

pytestmark = pytest.mark.gpu


def _static_rho_twice(w, parts, use_w):
    import torch
    from paper_1310_0930_gb300 import abi
    dev = torch.device("cuda", 0)
    cell = torch.from_numpy(np.ascontiguousarray(parts.cell, dtype=np.int32)).to(dev)
    off = torch.from_numpy(np.ascontiguousarray(parts.off, dtype=np.float32)).to(dev)
    wt = torch.from_numpy(np.ascontiguousarray(parts.w, dtype=np.float32)).to(dev)
    rho = torch.empty(w.n_cells, dtype=torch.float32, device=dev)
    grid = abi.pic_grid()
    grid.dim = w.dim
    for a in range(3):
        grid.n[a] = w.n[a] if a < w.dim else 1
    w_const = float(np.float32(w.density / w.ppc_total))  # the FP32 value the handle uses
    stream = torch.cuda.current_stream(dev)
    outs = []
    for _ in range(2):
        rho.fill_(float("nan"))
        rc = abi.lib().pic_charge_density_static(ctypes.byref(grid), w.order, -1.0, w_const, parts.n,
                                                 cell.data_ptr(), off.data_ptr(),
                                                 wt.data_ptr() if use_w else None, rho.data_ptr(),
                                                 stream.cuda_stream)
        assert rc == abi.PIC_OK, abi.pic_strerror(rc)
        torch.cuda.synchronize(dev)
        outs.append(rho.cpu().numpy().copy())
    return outs


@pytest.mark.parametrize("case", ["thermal_2d", "thermal_3d_cubic"])
def test_static_scratch_charge_matches_regular_path_twice(case):
    from paper_1310_0930_gb300.sim import Simulation
    if case == "thermal_2d":
        w = inputs.thermal_2d()
    else:
        w = inputs.thermal_3d(n=(16, 16, 16), order=3)
    parts = inputs.background(w)
    sim = Simulation(w)
    sim.load(parts)
    ref = sim.field("rho").reshape(-1).astype(np.float64)
    sim.close()
    orc = oracle_for(w, nthreads=2)
    load_oracle(orc, w, parts)
    ref64 = orc.charge()
    scale = np.max(np.abs(ref64))
    assert scale > 0
    assert np.max(np.abs(ref - ref64)) <= 1e-6 * scale
    for use_w in (False, True):
        for out in _static_rho_twice(w, parts, use_w):
            assert np.all(np.isfinite(out))
            assert np.max(np.abs(out.astype(np.float64) - ref)) <= 1e-6 * scale
            assert np.max(np.abs(out.astype(np.float64) - ref64)) <= 1e-6 * scale
