"""The autotuner's host logic on CPU, with a fake fleet and scripted timings (no GPU): every
candidate is timed once, those within 3 % of the fastest are timed again in turn and ranked by
their best time, the pick is cached under the fleet's key (and in the JSON cache file), and a
lone clear winner is not re-timed."""
import json

import numpy as np
import pytest

from paper_2410_14117_gb300 import autotune as A
from paper_2410_14117_gb300.autotune import Autotuner, LaunchConfig


class FakeSim:
    def __init__(self, n, types, vehicles):
        self.n, self.types, self.stream = n, types, None

    def randomize(self, *a, **k):
        pass

    def reset(self, *a, **k):
        pass

    def set_procedural_actions(self, *a, **k):
        pass

    def sync(self):
        return 0

    def close(self):
        pass


CANDS = [LaunchConfig("static", 64, 50, False), LaunchConfig("queue", 128, 50, True, 8),
         LaunchConfig("queue", 128, 100, True, 8), LaunchConfig("static", 32, 1000, True)]


def _tuner(monkeypatch, script, tmp_path=None):
    """script: cfg -> list of times (ms) returned by successive timings of that candidate."""
    calls = []

    def fake_time(self, sim, cfg, calls_per_rep, start, end):
        calls.append(cfg)
        return script[cfg].pop(0)

    monkeypatch.setattr(A, "Sim", FakeSim)
    monkeypatch.setattr(A.Autotuner, "_time_ms", fake_time)
    monkeypatch.setattr(A.torch.cuda, "Event", lambda **k: None)
    monkeypatch.setattr(A.torch.cuda, "get_device_name", lambda: "fake")
    path = str(tmp_path / "cache.json") if tmp_path else None
    return Autotuner(cache_path=path, candidates=CANDS, horizon=100, reps=2), calls


def test_refines_near_ties_by_best_time(monkeypatch, tmp_path):
    # first pass: chunk 50 looks fastest, chunk 100 within 3 %, the rest far behind; the re-timed
    # rounds show chunk 100 faster
    script = {CANDS[0]: [5.0], CANDS[1]: [1.00, 1.02, 1.01, 1.03],
              CANDS[2]: [1.02, 0.98, 0.99, 0.985], CANDS[3]: [3.0]}
    tuner, calls = _tuner(monkeypatch, script, tmp_path)
    res = tuner.measure(1000, np.zeros(1000, np.int32), [])
    assert [c for c, _ in res][:2] == [CANDS[2], CANDS[1]]
    # four first-pass timings, then three rounds over the two finalists only
    assert calls[:4] == CANDS and calls[4:] == [CANDS[1], CANDS[2]] * 3
    # the rate comes from the best time: 1000 envs x 100 sub-steps / 0.98 ms
    assert res[0][1] == pytest.approx(1000 * 100 / 0.98e-3)


def test_clear_winner_is_not_retimed_and_pick_is_cached(monkeypatch, tmp_path):
    script = {CANDS[0]: [5.0], CANDS[1]: [1.0], CANDS[2]: [1.5], CANDS[3]: [3.0]}
    tuner, calls = _tuner(monkeypatch, script, tmp_path)
    types = np.zeros(500, np.int32)
    best = tuner.pick(500, types, [])
    assert best == CANDS[1] and calls == CANDS
    assert tuner.pick(500, types, []) == best and len(calls) == 4  # cached: no new timings
    entry = json.load(open(tmp_path / "cache.json"))[tuner.key(500, types, [])]
    assert LaunchConfig(**entry["config"]) == best
    assert [LaunchConfig(**c) for c in entry["runner_up"]] == [CANDS[2], CANDS[3]]
