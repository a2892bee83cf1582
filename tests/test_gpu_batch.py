"""Batched form: several independent, uneven runs advanced together (one
launch per phase over all runs' tiles, CUDA-graph replay, persistent work
queue) give the same fields as each run advanced alone, and as the oracle."""
import numpy as np
import pytest

from gpu_helpers import FIELD_NAMES, load_oracle, oracle_for, rel_l2
from paper_1310_0930_gb300 import inputs
from paper_1310_0930_gb300.sim import Simulation

pytestmark = pytest.mark.gpu


def _runs():
    specs = [dict(nx=32, nz=160, ppc=(2, 2), density=0.004, a0=1.5, waist=8.0),
             dict(nx=64, nz=96, ppc=(3, 3), density=0.009, a0=3.0, waist=14.0),
             dict(nx=48, nz=224, ppc=(2, 4), density=0.002, a0=5.0, waist=10.0),
             dict(nx=16, nz=64, ppc=(4, 4), density=0.006, a0=1.0, waist=5.0)]
    runs = []
    for k, sp in enumerate(specs):
        w = inputs.lwfa_2d(steps=120, seed=40 + k, **sp)
        w.laser.fwhm = 6.0
        w.window.t0 = 20.0
        runs.append(w)
    return runs


def _fields(sim):
    return {n: sim.field(n) for n in FIELD_NAMES}


@pytest.mark.parametrize("persistent", [1, 2])
def test_batch_equals_individual_runs(persistent):
    runs = _runs()
    parts = [inputs.background(w) for w in runs]
    batch = Simulation(runs, tuning={"persistent": persistent})
    for r, p in enumerate(parts):
        batch.select(r)
        batch.load(p)
    batch.step(runs[0].steps)
    for r, (w, p) in enumerate(zip(runs, parts)):
        batch.select(r)
        fb = _fields(batch)
        nb = batch.diagnostics()
        single = Simulation(w)
        single.load(p)
        single.step(w.steps)
        fs = _fields(single)
        ns = single.diagnostics()
        single.close()
        assert nb["shifts"] == ns["shifts"] > 10
        assert nb["n_particles"] == ns["n_particles"]
        for n in FIELD_NAMES:
            assert rel_l2(fb[n], fs[n]) < 1e-5, (r, n)
    batch.close()


def test_batch_run_matches_oracle():
    runs = _runs()
    parts = [inputs.background(w) for w in runs]
    batch = Simulation(runs)
    for r, p in enumerate(parts):
        batch.select(r)
        batch.load(p)
    batch.step(runs[0].steps)
    r = 2
    w = runs[r]
    orc = oracle_for(w)
    load_oracle(orc, w, parts[r], extra=w.n[0] * w.ppc_total * 80)
    orc.step(w.steps)
    batch.select(r)
    worst = max(rel_l2(batch.field(n), orc.field(n)) for n in FIELD_NAMES)
    assert worst < 1e-4
    assert batch.diagnostics()["n_particles"] == orc.np
    batch.close()
