"""Autotuner for the step launch: picks envs-per-block, sub-steps per launch and the schedule
(static grid or work queue, its register budget and resident warps) for a fleet.

Candidates are timed with CUDA events on a scratch fleet with the same size and vehicle-type
layout as the target (randomised parameters, procedural commands), so tuning never touches the
target's state, parameters or actions.  Results are cached per (device, fleet size, type-run
signature, mass-matrix structure) in memory and, if ``cache_path`` is given, in a JSON file.
"""
from __future__ import annotations

import dataclasses
import hashlib
import json
import os

import numpy as np
import torch

from .sim import Sim


@dataclasses.dataclass(frozen=True)
class LaunchConfig:
    schedule: str          # "static" or "queue"
    envs_per_block: int    # static grid block size
    steps_per_launch: int  # static: sub-steps per launch; queue: sub-steps per unit (chunk)
    wide: bool = True      # 200-register diagonal-mass kernel (queue; static grid)
    warps_per_sm: int = 0  # queue: resident-warp cap (0 = as many as fit)

    def apply(self, sim: Sim, use_graph: bool = True):
        sim.set_launch(self.envs_per_block, self.steps_per_launch, use_graph)
        sim.set_schedule(self.schedule == "queue", self.wide, self.warps_per_sm)


DEFAULT_CANDIDATES = (
    # the static grid with the 128-register and the 200-register diagonal-mass kernel
    [LaunchConfig("static", epb, spl, wide) for wide in (False, True) for epb in (32, 64, 128, 256)
     for spl in (50, 1000)]
    + [LaunchConfig("queue", 128, ch, wide, wps)
       for wide, wps in ((False, 16), (False, 12), (True, 12), (True, 8))
       for ch in (25, 50, 100)]
)


def _signature(types: np.ndarray, vehicles, general: bool) -> str:
    runs = np.flatnonzero(np.diff(types)) if types.size > 1 else np.array([], dtype=np.int64)
    h = hashlib.sha1()
    h.update(types[np.r_[0, runs + 1]].tobytes())
    h.update(np.diff(np.r_[0, runs + 1, types.size]).astype(np.int64).tobytes())
    h.update(json.dumps([int(v.n_thr) for v in vehicles]).encode())
    h.update(b"general" if general else b"diag")
    return h.hexdigest()[:16]


class Autotuner:
    def __init__(self, cache_path: str | None = None, candidates=DEFAULT_CANDIDATES,
                 horizon: int = 300, reps: int = 3, k_per_call: int | None = None,
                 refine_rounds: int = 3):
        """``horizon`` sub-steps are timed per repetition, as one ``step(horizon)`` call, or as
        ``horizon // k_per_call`` calls of ``step(k_per_call)`` when the caller steps in small
        pieces (a policy loop): the best launch shape differs between the two."""
        self.cache_path = cache_path
        self.candidates = list(candidates)
        self.horizon = horizon
        self.reps = reps
        self.refine_rounds = refine_rounds
        self.k_per_call = k_per_call if k_per_call else horizon
        if not 1 <= self.k_per_call <= horizon:
            raise ValueError("need 1 <= k_per_call <= horizon")
        self.cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)

    def key(self, n_envs: int, types, vehicles, general: bool = False) -> str:
        dev = torch.cuda.get_device_name()
        sig = _signature(np.asarray(types, dtype=np.int32), vehicles, general)
        return f"{dev}|{n_envs}|{sig}|k{self.k_per_call}"

    def _time_ms(self, sim: Sim, cfg: LaunchConfig, calls: int, start, end) -> float:
        cfg.apply(sim)
        sim.step(self.k_per_call)  # warm-up (and graph capture)
        torch.cuda.synchronize()
        start.record(sim.stream)
        for _ in range(self.reps * calls):
            sim.step(self.k_per_call)
        end.record(sim.stream)
        torch.cuda.synchronize()
        return start.elapsed_time(end) / self.reps

    def measure(self, n_envs: int, types, vehicles, general: bool = False):
        """Time every candidate; returns [(config, env-steps/s)] sorted fastest first.  The
        candidates within 3 % of the fastest are timed again, in turn, ``refine_rounds`` times,
        and ranked by their best time: one short timing each leaves neighbours such as chunks
        of 50 and 100 sub-steps in an order that changes from run to run."""
        types = np.asarray(types, dtype=np.int32)
        sim = Sim(n_envs, types, vehicles)
        try:
            sim.randomize(7, 0.8, 1.2, 0.2, 0.3)
            if general:
                p = sim.get_params()
                p[:, 24:27] = 0.01
                sim.set_params(p)
            sim.reset()
            sim.set_procedural_actions(11, 10)
            start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            calls = self.horizon // self.k_per_call
            steps = n_envs * calls * self.k_per_call
            ms = {cfg: self._time_ms(sim, cfg, calls, start, end) for cfg in self.candidates}
            best = min(ms.values())
            finalists = sorted((c for c in ms if ms[c] <= 1.03 * best), key=ms.get)[:4]
            if len(finalists) > 1:
                for _ in range(self.refine_rounds):
                    for cfg in finalists:
                        ms[cfg] = min(ms[cfg], self._time_ms(sim, cfg, calls, start, end))
            sim.sync()
        finally:
            sim.close()
        out = [(cfg, steps / (t / 1e3)) for cfg, t in ms.items()]
        out.sort(key=lambda t: -t[1])
        return out

    def pick(self, n_envs: int, types, vehicles, general: bool = False) -> LaunchConfig:
        k = self.key(n_envs, types, vehicles, general)
        if k in self.cache:
            return LaunchConfig(**self.cache[k]["config"])
        res = self.measure(n_envs, types, vehicles, general)
        best, rate = res[0]
        self.cache[k] = {"config": dataclasses.asdict(best), "env_steps_per_s": rate,
                         "runner_up": [dataclasses.asdict(c) for c, _ in res[1:3]]}
        if self.cache_path:
            tmp = self.cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1)
            os.replace(tmp, self.cache_path)
        return best

    def tune(self, sim: Sim, vehicles, general: bool = False) -> LaunchConfig:
        """Pick the launch configuration for ``sim`` and apply it."""
        cfg = self.pick(sim.n, sim.types, vehicles, general)
        cfg.apply(sim)
        return cfg
