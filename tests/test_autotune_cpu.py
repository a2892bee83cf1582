"""Autotuner host logic (no GPU): coordinate-descent selection over the
compiled menu and the on-disk cache, with an injected timing function."""
import json

from paper_1310_0930_gb300 import autotune, inputs


def _cost(t):
    tile_cost = {(16, 16): 3.0, (8, 8): 2.0, (32, 32): 1.0}[tuple(t.get("tile", (16, 16)))]
    drift_cost = {1: 0.3, 2: 0.1, 3: 0.2}[t.get("drift", 2)]
    si_cost = {2: 0.5, 4: 0.2, 8: 0.4}[t.get("sort_interval", 4)]
    blk_cost = {128: 0.3, 256: 0.1, 512: 0.2}[t.get("block", 256)]
    per = {1: 0.05, 2: 0.0}[t.get("persistent", 1)]
    return tile_cost + drift_cost + si_cost + blk_cost + per


def test_search_picks_stagewise_optimum():
    best, trials = autotune.search(2, True, _cost)
    assert best == {"tile": (32, 32), "drift": 2, "sort_interval": 4, "block": 256, "persistent": 2}
    assert len(trials) == 5 + 3 + 3 + 2


def test_tune_caches_results(tmp_path):
    path = str(tmp_path / "cache.json")
    calls = []

    def measure(t):
        calls.append(t)
        return _cost(t)

    w = inputs.thermal_2d(n=(64, 64))
    t1 = autotune.tune(w, measure=measure, cache_path=path)
    n = len(calls)
    assert n == 5 + 3 + 3
    t2 = autotune.tune(w, measure=measure, cache_path=path)
    assert t1 == t2 and len(calls) == n  # second call served from the cache
    data = json.load(open(path))
    assert autotune.key_for(w) in data
    # a different workload bucket is tuned separately
    autotune.tune(inputs.thermal_2d(n=(512, 512)), measure=measure, cache_path=path)
    assert len(calls) == 2 * n


def test_keys_separate_dims_orders_and_batches():
    a = autotune.key_for(inputs.thermal_2d())
    b = autotune.key_for(inputs.thermal_2d(order=3))
    c = autotune.key_for([inputs.thermal_2d(), inputs.thermal_2d()])
    d = autotune.key_for(inputs.thermal_3d())
    assert len({a, b, c, d}) == 4
