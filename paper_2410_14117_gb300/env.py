"""Gym-style vectorised environment over the fused task step.

The paper's four tasks (§EXPERIMENTS: station keeping, circle, helix and lemniscate tracking)
are offered in a Gym-style format: a policy sees the observation of Eq. 2, sets one throttle per
thruster (the action space of Eq. 3) and is scored by the position error of Eq. 4.
``MarineEnv`` keeps a whole fleet of such environments on the GPU.  ``step`` is one library call
(mg_env_step): the actions are clamped into the library's resident one-segment schedule, every
env advances ``sub_steps`` RK4 sub-steps (the paper's sub-simulation steps within one simulation
step), and the observation, the reward and the auto-reset of finished episodes are fused into
the last launch.  The reward is the negative position error: the paper names the error the tasks
are judged by, not its reward weights.

Every env's reference path starts within ``spawn_radius`` of the origin, where a reset puts
the vehicle; each env has its own phase on its path.
"""
from __future__ import annotations

import math

import numpy as np
import torch

import ctypes

from . import _lib
from . import inputs as I
from ._lib import MGError
from .sim import Sim

# mg.h MG_TASK_*
TASKS = {"station": 0, "circle": 1, "helix": 2, "lemniscate": 3}


def task_centres(task: str, n_envs: int, radius: float, seed: int,
                 spawn_radius: float = 0.5) -> np.ndarray:
    """Centres and phases [n_envs, 4] = (cx, cy, cz, phi0) that put every env's reference at
    t = 0 within spawn_radius of the origin (uniform in the ball), at a uniform random phase."""
    if task not in TASKS:
        raise ValueError(f"unknown task {task!r}; one of {sorted(TASKS)}")
    g = np.random.default_rng(seed)
    phase = g.uniform(0.0, 2.0 * math.pi, n_envs)
    c = np.zeros((n_envs, 4))
    c[:, 3] = phase
    if task in ("circle", "helix"):
        c[:, 0] = -radius * np.cos(phase)
        c[:, 1] = -radius * np.sin(phase)
    elif task == "lemniscate":
        den = 1.0 + np.sin(phase) ** 2
        c[:, 0] = -radius * np.cos(phase) / den
        c[:, 1] = -radius * np.sin(phase) * np.cos(phase) / den
    # offsets uniform in the ball of radius spawn_radius
    d = g.normal(size=(n_envs, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    c[:, :3] += d * (spawn_radius * g.uniform(0.0, 1.0, (n_envs, 1)) ** (1.0 / 3.0))
    return c


class MarineEnv:
    """``n_envs`` environments of one task; ``vehicle`` is a vehicle type for all of them or a
    per-env sequence of types (a mixed fleet; actions then have the largest thruster count, and
    entries past an env's own count are ignored).

    reset() -> obs [n, obs_dim];  step(actions [n, n_thr]) -> (obs, reward [n], done [n] bool,
    {"episode_error": [n]}).  All four live on the GPU in buffers the next call overwrites
    (done is a bool view of the step's flags).  Throttles are clamped to [-1, 1].  An
    episode ends when the position error exceeds ``max_error``, after ``episode_steps``
    sub-steps, or on a non-finite state; the env is then reset inside the step and its returned
    observation is the new episode's first.  tune: time the launch shapes for calls of
    sub_steps sub-steps first (a few seconds; at 1,024-65,536 envs the default shape measured
    within 8 % of the tuned one, either way).  The fleet runs on torch's current stream at
    construction.
    """

    def __init__(self, n_envs: int, task: str = "circle", vehicle=1, sub_steps: int = 10,
                 seed: int = 0, dt: float = 0.01, lo: float = 0.8, hi: float = 1.2,
                 current_sigma: float = 0.2, nu0_sigma: float = 0.0, radius: float = 2.0,
                 omega: float = 0.3, vz: float = 0.1, psi_r: float = 0.0, lookahead: int = 4,
                 lookahead_dt: float = 0.5, max_error: float = 3.0, episode_steps: int = 1000,
                 spawn_radius: float = 0.5, vehicles=None, tune: bool = False):
        if task not in TASKS:
            raise ValueError(f"unknown task {task!r}; one of {sorted(TASKS)}")
        if sub_steps < 1:
            raise ValueError("sub_steps must be >= 1")
        self.vehicles = list(vehicles) if vehicles is not None else I.fleet_vehicles()
        self.n, self.k, self.task = int(n_envs), int(sub_steps), task
        types = (np.full(self.n, vehicle, dtype=np.int32) if np.ndim(vehicle) == 0
                 else np.asarray(vehicle, dtype=np.int32))
        if types.shape != (self.n,) or types.min() < 0 or types.max() >= len(self.vehicles):
            raise ValueError("vehicle: a type index, or one per env, in range")
        self.types = types
        self.n_thr = max(int(self.vehicles[t].n_thr) for t in np.unique(types))
        sim = Sim(self.n, types, self.vehicles)
        self.sim = sim
        sim.set_timestep(dt)
        if tune:  # launch shape timed for calls of sub_steps sub-steps (on a scratch fleet)
            from .autotune import Autotuner
            Autotuner(horizon=10 * self.k, reps=2, k_per_call=self.k).tune(sim, self.vehicles)
        if self.n_thr == 6:  # every env has 6 thrusters: unpadded throttle rows
            sim.set_action_width(6)
        sim.randomize(seed, lo, hi, current_sigma, nu0_sigma)
        sim.reset()
        self.centres = torch.tensor(task_centres(task, self.n, radius, seed, spawn_radius),
                                    dtype=torch.float32, device=sim.device)
        self._task_args = dict(radius=radius, omega=omega, vz=vz, psi_r=psi_r,
                               lookahead=lookahead, lookahead_dt=lookahead_dt,
                               max_error=max_error, episode_steps=episode_steps)
        sim.set_task(TASKS[task], self.centres, **self._task_args)
        self.obs_dim = sim.obs_dim
        self.action_dim = self.n_thr
        dev = sim.device
        self._obs = torch.empty((self.n, self.obs_dim), dtype=torch.float32, device=dev)
        self._rew = torch.empty(self.n, dtype=torch.float32, device=dev)
        self._err = torch.empty(self.n, dtype=torch.float32, device=dev)
        self._done = torch.zeros(self.n, dtype=torch.uint8, device=dev)
        self._ep = torch.zeros(self.n, dtype=torch.float32, device=dev)
        self._lib = _lib.load()
        p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
        self._step_outs = (p(self._obs), p(self._rew), p(self._done), p(self._ep))
        self._obs_outs = (p(self._obs), p(self._err), p(self._done), p(self._ep))
        self._info = {"episode_error": self._ep}

    def _check(self, st, where):
        if st != 0:
            raise MGError(st, where, self._lib.mg_last_error().decode(errors="replace"))

    def reset(self):
        """Start a new episode in every env (state reset, episode clocks and error sums back to
        zero); returns the observation."""
        self.sim.reset()
        self.sim.set_task(TASKS[self.task], self.centres, **self._task_args)
        self._check(self._lib.mg_task_step(self.sim._h, 0, *self._obs_outs), "mg_task_step")
        return self._obs

    def step(self, actions):
        a = actions
        if not (isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.float32
                and a.is_contiguous()):
            a = torch.as_tensor(a, dtype=torch.float32).to(self._obs.device).contiguous()
        if tuple(a.shape) != (self.n, self.n_thr):
            raise ValueError(f"actions must be [{self.n}, {self.n_thr}]")
        self._check(self._lib.mg_env_step(self.sim._h, self.k, ctypes.c_void_p(a.data_ptr()),
                                          *self._step_outs), "mg_env_step")
        return self._obs, self._rew, self._done.view(torch.bool), self._info

    def close(self):
        if self.sim is not None:
            self.sim.close()
            self.sim = None
