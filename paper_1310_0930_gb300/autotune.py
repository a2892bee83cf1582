"""Autotuner for the launch configuration of the EM-PIC timestep.

Chooses, for a set of runs (one run or a batch), the tile geometry and drift
allowance from the compiled menu, the sort interval, the threads per tile
CTA (the knob that sets how many threads share a tile's particles) and, for
batches, persistent work-queue scheduling versus one CTA per tile.  The
search is coordinate descent in that order on a short trial of the actual
workload; results are cached in a JSON file keyed by dimension, shape order,
particles per cell, a power-of-two bucket of the total cell count and the
batch size.  The timing function can be injected (the CPU tests do).
"""
from __future__ import annotations

import json
import math
import os
import threading
from typing import Callable, Optional

TILES = {2: [((16, 16), 2), ((8, 8), 1), ((32, 32), 2), ((16, 16), 1), ((16, 16), 3)],
         3: [((8, 8, 8), 1), ((8, 8, 8), 2)]}
SORT_INTERVALS = [2, 4, 8]
BLOCKS = {2: [256, 512, 128], 3: [512, 256]}

_lock = threading.Lock()


def default_cache_path() -> str:
    return os.environ.get("PIC_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "pic_gb300_autotune.json"))


def key_for(workloads) -> str:
    ws = workloads if isinstance(workloads, (list, tuple)) else [workloads]
    dim, order = ws[0].dim, ws[0].order
    cells = sum(w.n_cells for w in ws)
    ppc = max(w.ppc_total for w in ws)
    return "d%d_p%d_ppc%d_cells2^%d_runs%d" % (dim, order, ppc, int(round(math.log2(max(cells, 1)))), len(ws))


def candidates(dim: int, batched: bool):
    """Coordinate-descent stages: each is a list of partial tunings."""
    stages = [[{"tile": t, "drift": d} for t, d in TILES[dim]],
              [{"sort_interval": s} for s in SORT_INTERVALS],
              [{"block": b} for b in BLOCKS[dim]]]
    if batched:
        stages.append([{"persistent": 1}, {"persistent": 2}])
    return stages


def search(dim: int, batched: bool, measure: Callable[[dict], float]):
    """Coordinate descent: returns (best tuning, trials [(tuning, cost)])."""
    best: dict = {}
    trials = []
    for stage in candidates(dim, batched):
        scored = []
        for opt in stage:
            t = dict(best)
            t.update(opt)
            cost = measure(t)
            trials.append((t, cost))
            scored.append((cost, t))
        scored.sort(key=lambda x: x[0])
        best = scored[0][1]
    return best, trials


def gpu_measure(workloads, loader: Callable, steps: int = 6, warmup: int = 2):
    """Seconds per particle-step of a short trial through the C ABI."""
    from .sim import Simulation

    def measure(tuning: dict) -> float:
        sim = Simulation(workloads, tuning=tuning)
        try:
            n = loader(sim)
            sim.step(warmup)
            sim.sync()
            sim.profile_begin(steps)
            sim.step(steps)
            phases, _ = sim.profile_end()
            return sum(phases.values()) / 1e3 / max(1, n * steps)
        finally:
            sim.close()
    return measure


def _normal(t: dict) -> dict:
    t = dict(t)
    if "tile" in t:
        t["tile"] = tuple(t["tile"])
    return t


def tune(workloads, loader: Optional[Callable] = None, *, measure: Optional[Callable[[dict], float]] = None,
         cache_path: Optional[str] = None, refresh: bool = False) -> dict:
    """Best tuning for `workloads` (cached).  `loader(sim)` loads the
    particles into a Simulation and returns their count."""
    ws = workloads if isinstance(workloads, (list, tuple)) else [workloads]
    key = key_for(ws)
    path = cache_path or default_cache_path()
    with _lock:
        cache = {}
        if os.path.exists(path):
            try:
                with open(path) as f:
                    cache = json.load(f)
            except (OSError, ValueError):
                cache = {}
        if key in cache and not refresh:
            return _normal(cache[key]["tuning"])
    if measure is None:
        if loader is None:
            raise ValueError("tune() needs a loader or a measure function")
        measure = gpu_measure(workloads, loader)
    best, trials = search(ws[0].dim, len(ws) > 1, measure)
    with _lock:
        cache[key] = {"tuning": best, "trials": [[t, c] for t, c in trials]}
        d = os.path.dirname(path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return _normal(best)
