"""Launch autotuner: it times real candidates on a scratch fleet, leaves the target untouched,
caches per (device, fleet size, type layout, call size) in memory and on disk, and whatever it
picks, results are bit-identical to the default launch."""
import json

import numpy as np
import pytest
import torch

from paper_2410_14117_gb300 import inputs as I
from paper_2410_14117_gb300.autotune import Autotuner, LaunchConfig
from paper_2410_14117_gb300.sim import Sim

from _helpers import vehicles

CANDS = [LaunchConfig("static", 64, 50), LaunchConfig("static", 128, 1),
         LaunchConfig("queue", 128, 25, True, 8), LaunchConfig("queue", 128, 50, False, 16)]


def _run(types, vs, cfg=None):
    sim = Sim(len(types), types, vs)
    if cfg is not None:
        cfg.apply(sim)
    sim.randomize(4, 0.8, 1.2, 0.2, 0.3)
    sim.reset()
    sim.set_procedural_actions(6, 10)
    for _ in range(6):
        sim.step(10)
    out = sim.get_state().cpu()
    sim.close()
    return out


@pytest.mark.gpu
def test_pick_caches_and_keeps_results(tmp_path):
    vs = vehicles()
    n = 2500
    types = I.mixed_fleet(2, n, max_group=700)
    path = str(tmp_path / "tune.json")
    tuner = Autotuner(cache_path=path, candidates=CANDS, horizon=40, reps=1, k_per_call=10)
    res = tuner.measure(n, types, vs)
    assert {c for c, _ in res} == set(CANDS)
    assert all(r > 0 for _, r in res) and res[0][1] >= res[-1][1]
    best = tuner.pick(n, types, vs)
    assert best in CANDS
    with open(path) as f:
        cache = json.load(f)
    (key, entry), = cache.items()
    assert key.endswith("|k10") and LaunchConfig(**entry["config"]) == best
    # a fresh tuner reads the cache instead of timing again
    again = Autotuner(cache_path=path, candidates=[], horizon=40, reps=1, k_per_call=10)
    assert again.pick(n, types, vs) == best
    # another call size is another key
    assert Autotuner(candidates=[], horizon=40, k_per_call=20).key(n, types, vs) != key
    torch.testing.assert_close(_run(types, vs, best), _run(types, vs), rtol=0, atol=0)


def test_k_per_call_validated():
    with pytest.raises(ValueError):
        Autotuner(horizon=10, k_per_call=20)
