"""Serving rollouts with continuous batching.

``Pool`` binds the native job pool (mg_pool_*): jobs of different sizes, vehicle types and
horizons share one arena and advance together, one launch per tick.  ``Server`` is the request
loop on top: requests arrive over time, wait in a FIFO queue until the HBM budget and a free
arena range admit them, run as slots of the shared persistent launches, and leave when their
horizon is done; the loop reports p50/p99 latency (arrival to result) and env-steps/s.  The same
loop in ``mode="serial"`` runs one job at a time, which is the baseline.
"""
from __future__ import annotations

import collections
import ctypes
import dataclasses
import time

import numpy as np
import torch

from ._lib import (MG_NSTATE, MG_NTRAJ, MG_NXPARAM, JobSpec, MGError, Ranges, ServerConfig,
                   VehicleParams, call)
from .sim import _ptr, vehicle_struct

# Device bytes per env held by the pool arena (state planes, parameter planes and records,
# type, flags, episode counter), used for budget accounting.
ARENA_BYTES_PER_ENV = 5 * 16 + 4 + 8 * 16 + 8 + 5 * 16 + 4 + 35 * 4 + 4 + 4 + 4


class Pool:
    def __init__(self, capacity_envs: int, vehicles, stream=None):
        self._h = None
        arr = (VehicleParams * len(vehicles))(*[vehicle_struct(v) for v in vehicles])
        h = ctypes.c_void_p()
        call("mg_pool_create", int(capacity_envs), arr, len(vehicles), ctypes.byref(h))
        self._h = h
        self.capacity = int(capacity_envs)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        call("mg_pool_set_stream", self._h, ctypes.c_void_p(self.stream.cuda_stream))

    def admit(self, n_envs, vehicle_type, horizon, param_seed, cmd_seed, hold=10, traj=None,
              lo=0.8, hi=1.2, current_sigma=0.2, nu0_sigma=0.3, rg_halfwidth=0.0, xh=None):
        """Job id, or None when no free range is large enough.  xh: the job's off-diagonal
        added mass and linear damping, float32 [n_envs, MG_NXPARAM] (host or device), or None."""
        spec = JobSpec(int(n_envs), int(vehicle_type), int(hold), int(horizon), 0,
                       int(param_seed), int(cmd_seed),
                       Ranges(lo, hi, current_sigma, nu0_sigma, 0, rg_halfwidth))
        jid = ctypes.c_int32()
        tp = _ptr(traj) if traj is not None else None
        if xh is None:
            st = call("mg_pool_admit", self._h, ctypes.byref(spec), tp, ctypes.byref(jid),
                      ok=(0, 2))
        else:
            if tuple(xh.shape) != (int(n_envs), MG_NXPARAM) or xh.dtype not in (
                    torch.float32, np.float32):
                raise ValueError(f"xh must be float32 [{int(n_envs)}, {MG_NXPARAM}]")
            st = call("mg_pool_admit_offdiag", self._h, ctypes.byref(spec), tp, _ptr(xh),
                      ctypes.byref(jid), ok=(0, 2))
        return None if st == 2 else jid.value

    def tick(self, k: int) -> int:
        n = ctypes.c_int32()
        call("mg_pool_tick", self._h, int(k), ctypes.byref(n))
        return n.value

    def progress(self, job_id: int):
        d, h = ctypes.c_int32(), ctypes.c_int32()
        call("mg_pool_job_progress", self._h, int(job_id), ctypes.byref(d), ctypes.byref(h))
        return d.value, h.value

    def job_state(self, job_id: int, n_envs: int):
        out = torch.empty((n_envs, MG_NSTATE), dtype=torch.float32, device=self.device)
        call("mg_pool_get_job_state", self._h, int(job_id), _ptr(out))
        return out

    def release(self, job_id: int):
        call("mg_pool_release", self._h, int(job_id))

    def info(self):
        f, b, j = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        call("mg_pool_info", self._h, ctypes.byref(f), ctypes.byref(b), ctypes.byref(j))
        return {"free_envs": f.value, "largest_free_range": b.value, "jobs": j.value}

    def sync(self):
        call("mg_pool_sync", self._h)

    def close(self):
        if self._h is not None:
            from ._lib import load
            load().mg_pool_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclasses.dataclass
class Request:
    arrival_s: float
    n_envs: int
    horizon: int
    vehicle: int
    param_seed: int
    cmd_seed: int
    hold: int = 10
    admitted_s: float = float("nan")
    done_s: float = float("nan")
    job_id: int = -1
    traj: object = None
    final_state: object = None
    xh: object = None  # off-diagonal added mass and damping, float32 [n_envs, MG_NXPARAM], or None

    @property
    def latency_s(self):
        return self.done_s - self.arrival_s


def traj_bytes(r: Request) -> int:
    return r.horizon * MG_NTRAJ * 4 * r.n_envs


class Server:
    """Continuous-batching rollout server over one Pool.

    budget_bytes bounds the device memory of resident jobs (their arena share plus trajectory
    records); capacity_envs sizes the arena; k is the sub-steps per tick (chunk size)."""

    def __init__(self, vehicles, budget_bytes: float = 120e9, capacity_envs: int = 4 << 20,
                 k: int = 50, record: bool = True, keep_results: bool = False,
                 wait_timeout_s: float = 30.0, pool=None, event=None):
        """wait_timeout_s bounds every host wait on the device (a tick that has not completed by
        then raises TimeoutError instead of blocking forever); pool and event (a factory of
        objects with record(stream) and query()) replace the device pool and CUDA events, for
        host-side tests."""
        self.vehicles = vehicles
        self.budget = float(budget_bytes)
        self.k = int(k)
        self.record = record
        self.keep_results = keep_results
        self.wait_timeout_s = float(wait_timeout_s)
        self.pool = pool if pool is not None else Pool(capacity_envs, vehicles)
        self.event = event if event is not None else torch.cuda.Event
        self.stream = self.pool.stream
        self.used = self.pool.capacity * ARENA_BYTES_PER_ENV
        self.peak_used = self.used
        if self.used > self.budget:
            raise ValueError("the arena alone exceeds the budget")

    def close(self):
        self.pool.close()

    def _traj_buffer(self, r):
        dev = getattr(self.pool, "device", None)
        return torch.empty((r.horizon, MG_NTRAJ, r.n_envs), dtype=torch.float32, device=dev)

    def run(self, requests, mode: str = "batched", realtime: bool = True, max_inflight: int = 2):
        """Serve ``requests`` (sorted by arrival_s); returns (served requests, stats)."""
        reqs = sorted(requests, key=lambda r: r.arrival_s)
        pool, k = self.pool, self.k
        room = self.budget - pool.capacity * ARENA_BYTES_PER_ENV
        for r in reqs:
            if r.n_envs > pool.capacity or (self.record and traj_bytes(r) > room):
                raise ValueError(f"request of {r.n_envs} envs x {r.horizon} sub-steps can never "
                                 "be admitted (arena capacity or budget too small)")
        queue = collections.deque()
        running = {}
        inflight = collections.deque()
        done = []
        nxt = 0
        queue_depth = []
        t0 = time.perf_counter()
        offset = 0.0 if realtime else None

        def now():
            return time.perf_counter() - t0

        def finish(ev, finishing):
            start = time.perf_counter()
            deadline = start + self.wait_timeout_s
            while not ev.query():  # polled, never an unbounded wait
                t_poll = time.perf_counter()
                if t_poll > deadline:
                    raise TimeoutError(f"a serving tick did not complete within "
                                       f"{self.wait_timeout_s} s")
                # spin for the first millisecond (a sleep's wake-up delay would add to the
                # job's latency), then poll every 20 us
                if t_poll - start > 1e-3:
                    time.sleep(20e-6)
            t = now()
            for jid in finishing:
                r = running.pop(jid)
                r.done_s = t
                if self.keep_results:
                    r.final_state = pool.job_state(jid, r.n_envs)
                pool.release(jid)
                self.used -= traj_bytes(r) if self.record else 0
                if not self.keep_results:
                    r.traj = None
                done.append(r)

        while nxt < len(reqs) or queue or running or inflight:
            t = now()
            while nxt < len(reqs) and (not realtime or reqs[nxt].arrival_s <= t):
                if not realtime:
                    reqs[nxt].arrival_s = t
                queue.append(reqs[nxt])
                nxt += 1
            queue_depth.append(len(queue))
            # FIFO admission while the budget and a free range allow
            while queue and (mode == "batched" or not running):
                r = queue[0]
                need = traj_bytes(r) if self.record else 0
                if self.used + need > self.budget:
                    break
                traj = (self._traj_buffer(r) if self.record else None)
                jid = pool.admit(r.n_envs, r.vehicle, r.horizon, r.param_seed, r.cmd_seed,
                                 r.hold, traj, xh=r.xh)
                if jid is None:
                    break
                r.job_id, r.traj, r.admitted_s = jid, traj, now()
                running[jid] = r
                self.used += need
                self.peak_used = max(self.peak_used, self.used)
                queue.popleft()
            if running:
                live = [j for j in running if pool.progress(j)[0] < running[j].horizon]
                if live:
                    pool.tick(k)
                finishing = [j for j in running
                             if pool.progress(j)[0] >= running[j].horizon and
                             not any(j in f for _, f in inflight)]
                ev = self.event()
                ev.record(self.stream)
                inflight.append((ev, finishing))
                while inflight and (len(inflight) > max_inflight or inflight[0][0].query()):
                    finish(*inflight.popleft())
            elif inflight:
                finish(*inflight.popleft())
            elif nxt < len(reqs):
                wait = reqs[nxt].arrival_s - now()
                if wait > 0:
                    time.sleep(min(wait, 0.0005))
        makespan = max(r.done_s for r in done) - min(r.arrival_s for r in done)
        lat = np.array([r.latency_s for r in done])
        steps = float(sum(r.n_envs * r.horizon for r in done))
        stats = {"mode": mode, "jobs": len(done), "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                 "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                 "mean_ms": 1e3 * float(lat.mean()), "env_steps_per_s": steps / makespan,
                 "makespan_s": makespan, "env_steps": steps,
                 "max_queue_depth": int(max(queue_depth) if queue_depth else 0),
                 "k": k}
        return done, stats


def requests_from_specs(specs, hold: int = 10):
    """Requests from inputs.serving_jobs() specs."""
    return [Request(arrival_s=s.arrival_s, n_envs=s.n_envs, horizon=s.horizon,
                    vehicle=s.vehicle, param_seed=s.param_seed, cmd_seed=s.cmd_seed, hold=hold)
            for s in specs]


class NativeServer:
    """The request loop of ``Server`` run natively (mg_server_*): admission, ticks and
    completion handling happen inside the library; the host submits requests when they arrive
    and calls one poll per round.  Same arguments, results and statistics as ``Server``."""

    def __init__(self, vehicles, budget_bytes: float = 120e9, capacity_envs: int = 4 << 20,
                 k: int = 50, record: bool = True, keep_results: bool = False,
                 wait_timeout_s: float = 30.0, max_inflight: int = 2):
        self.vehicles = vehicles
        self.budget = float(budget_bytes)
        self.k = int(k)
        self.record = record
        self.keep_results = keep_results
        self.wait_timeout_s = float(wait_timeout_s)
        self.max_inflight = int(max_inflight)
        self.pool = Pool(capacity_envs, vehicles)
        self.arena_bytes = self.pool.capacity * ARENA_BYTES_PER_ENV
        if self.arena_bytes > self.budget:
            raise ValueError("the arena alone exceeds the budget")
        self.peak_used = self.arena_bytes
        self._servers = {}  # mode -> native server, kept so its record memory pool stays warm

    def _server(self, mode):
        if mode not in self._servers:
            cfg = ServerConfig(self.budget - self.arena_bytes, self.k, self.max_inflight,
                               1 if self.record else 0, 1 if mode == "serial" else 0,
                               1 if self.keep_results else 0, 0, self.wait_timeout_s)
            h = ctypes.c_void_p()
            call("mg_server_create", self.pool._h, ctypes.byref(cfg), ctypes.byref(h))
            self._servers[mode] = h
        return self._servers[mode]

    def close(self):
        for h in self._servers.values():
            call("mg_server_destroy", h)
        self._servers = {}
        self.pool.close()

    def run(self, requests, mode: str = "batched", realtime: bool = True):
        """Serve ``requests`` (sorted by arrival_s); returns (served requests, stats)."""
        reqs = sorted(requests, key=lambda r: r.arrival_s)
        room = self.budget - self.arena_bytes
        for r in reqs:
            if r.n_envs > self.pool.capacity or (self.record and traj_bytes(r) > room):
                raise ValueError(f"request of {r.n_envs} envs x {r.horizon} sub-steps can never "
                                 "be admitted (arena capacity or budget too small)")
        h = self._server(mode)
        d = [ctypes.c_double() for _ in range(3)]

        def clock():
            call("mg_server_info", h, ctypes.byref(d[0]), None, None)
            return d[0].value

        tickets = {}
        counts = [ctypes.c_int32() for _ in range(3)]
        queue_depth = []
        nxt = 0
        t_start = clock()
        while True:
            t = clock() - t_start
            while nxt < len(reqs) and (not realtime or reqs[nxt].arrival_s <= t):
                r = reqs[nxt]
                if not realtime:
                    r.arrival_s = t
                spec = JobSpec(int(r.n_envs), int(r.vehicle), int(r.hold), int(r.horizon), 0,
                               int(r.param_seed), int(r.cmd_seed),
                               Ranges(0.8, 1.2, 0.2, 0.3, 0))
                tk = ctypes.c_int64()
                if r.xh is None:
                    call("mg_server_submit", h, ctypes.byref(spec), ctypes.byref(tk))
                else:
                    call("mg_server_submit_offdiag", h, ctypes.byref(spec), _ptr(r.xh),
                         ctypes.byref(tk))
                tickets[tk.value] = r
                nxt += 1
            call("mg_server_poll", h, *[ctypes.byref(c) for c in counts])
            queued, running, inflight = (c.value for c in counts)
            queue_depth.append(queued)
            if queued or running or inflight:
                continue
            if nxt == len(reqs):
                break
            wait = reqs[nxt].arrival_s - (clock() - t_start)
            if wait > 3e-4:
                time.sleep(wait - 2e-4)  # then spin to the arrival
        done = []
        for tk, r in tickets.items():
            call("mg_server_job", h, tk, None, ctypes.byref(d[1]), ctypes.byref(d[2]))
            r.job_id = tk
            r.admitted_s, r.done_s = d[1].value - t_start, d[2].value - t_start
            if self.keep_results:
                r.final_state = torch.empty((r.n_envs, MG_NSTATE), dtype=torch.float32,
                                            device=self.pool.device)
                r.traj = (torch.empty((r.horizon, MG_NTRAJ, r.n_envs), dtype=torch.float32,
                                      device=self.pool.device) if self.record else None)
                call("mg_server_job_result", h, tk, _ptr(r.final_state),
                     _ptr(r.traj) if r.traj is not None else None)
                call("mg_server_release", h, tk)
            done.append(r)
        call("mg_server_info", h, None, None, ctypes.byref(d[0]))
        self.peak_used = max(self.peak_used, self.arena_bytes + d[0].value)
        makespan = max(r.done_s for r in done) - min(r.arrival_s for r in done)
        lat = np.array([r.latency_s for r in done])
        steps = float(sum(r.n_envs * r.horizon for r in done))
        stats = {"mode": mode, "jobs": len(done), "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                 "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                 "mean_ms": 1e3 * float(lat.mean()), "env_steps_per_s": steps / makespan,
                 "makespan_s": makespan, "env_steps": steps,
                 "max_queue_depth": int(max(queue_depth) if queue_depth else 0),
                 "k": self.k}
        return done, stats
