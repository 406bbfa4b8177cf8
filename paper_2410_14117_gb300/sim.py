"""``Sim``: a fleet of vehicles advanced by the extended Fossen equation (§METHOD, Eq. 1) on the
GPU.  A thin wrapper of the C ABI: every computation runs in libmg.so's kernels; PyTorch only
provides device memory and the stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import (MG_MAX_THR, MG_NPARAM, MG_NSTATE, MG_NTRAJ, MG_NXPARAM, MG_RANDOMIZE_ASYNC,
                   MGError, Ranges, TaskSpec, VehicleParams, call)

__all__ = ["Sim", "vehicle_struct", "MGError"]


def vehicle_struct(v) -> VehicleParams:
    """Convert a vehicle definition (``params`` [35] array, ``n_thr``, ``r`` [8,3], ``d`` [8,3]
    — e.g. ``inputs.bluerov2()``) to the C struct."""
    p = np.asarray(v.params, dtype=np.float64)
    s = VehicleParams()
    s.m, s.Ixx, s.Iyy, s.Izz = p[0], p[1], p[2], p[3]
    for i in range(6):
        s.MA[i], s.Dl[i], s.Dq[i] = p[4 + i], p[10 + i], p[16 + i]
    s.W, s.B = p[22], p[23]
    for i in range(3):
        s.rg[i], s.rb[i] = p[24 + i], p[27 + i]
    s.kT, s.tau_m = p[30], p[31]
    s.n_thr = int(v.n_thr)
    r = np.asarray(v.r, dtype=np.float64)
    d = np.asarray(v.d, dtype=np.float64)
    for i in range(MG_MAX_THR):
        for j in range(3):
            s.r[i][j] = r[i, j]
            s.d[i][j] = d[i, j]
    return s


def _ptr(t) -> ctypes.c_void_p:
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(t.ctypes.data)
    raise TypeError(f"expected a torch tensor or numpy array, got {type(t)}")


def _check(t, shape, dtype):
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    if isinstance(t, torch.Tensor) and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    if isinstance(t, np.ndarray) and t.dtype != np.dtype(str(dtype).split(".")[-1]):
        raise ValueError(f"expected {dtype}, got {t.dtype}")


class Sim:
    """A fleet of ``n_envs`` vehicles on the current CUDA device.

    ``vehicle_types``: int array [n_envs] indexing ``vehicles`` (a list of vehicle definitions).
    The sim runs on ``stream`` (default: torch's current stream at construction).
    """

    def __init__(self, n_envs: int, vehicle_types, vehicles, stream=None):
        self._h = None
        types = np.ascontiguousarray(np.broadcast_to(np.asarray(vehicle_types, dtype=np.int32),
                                                     (n_envs,)))
        arr = (VehicleParams * len(vehicles))(*[vehicle_struct(v) for v in vehicles])
        h = ctypes.c_void_p()
        call("mg_create", n_envs, types.ctypes.data, arr, len(vehicles), ctypes.byref(h))
        self._h = h
        self.n = int(n_envs)
        self.types = types
        self.n_thr = np.array([int(vehicles[t].n_thr) for t in types], dtype=np.int32)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.act_w = MG_MAX_THR
        self.set_stream(stream if stream is not None else torch.cuda.current_stream())

    # ------------------------------------------------------------------ configuration
    def set_stream(self, stream):
        self.stream = stream
        call("mg_set_stream", self._h, ctypes.c_void_p(stream.cuda_stream))

    def set_env_id_offset(self, offset: int):
        call("mg_set_env_id_offset", self._h, int(offset))

    def set_model_flags(self, flags: int):
        call("mg_set_model_flags", self._h, int(flags))

    def set_timestep(self, dt: float):
        call("mg_set_timestep", self._h, float(dt))

    def set_launch(self, envs_per_block: int = 128, steps_per_launch: int = 50,
                   use_graph: bool = True):
        call("mg_set_launch", self._h, int(envs_per_block), int(steps_per_launch),
             1 if use_graph else 0)

    def set_schedule(self, work_queue: bool = False, wide: bool = True, warps_per_sm: int = 0):
        """Static grid (default) or the work-queue schedule (see mg_set_schedule)."""
        call("mg_set_schedule", self._h, 1 if work_queue else 0, 1 if wide else 0,
             int(warps_per_sm))

    def set_wait_limit(self, polls: int = 0):
        """Bound on each work-queue wait in polls of ~128 ns (0: the default; see
        mg_set_wait_limit)."""
        call("mg_set_wait_limit", self._h, int(polls))

    def set_adjoint_mode(self, mode: int = 0):
        """Backward kernel of the adjoint: 0 by fleet size, 1 one warp per 32 envs, 2 a
        producer and a consumer warp per 32 envs (see mg_set_adjoint_mode)."""
        call("mg_set_adjoint_mode", self._h, int(mode))

    def kernel_info(self) -> dict:
        r, t, l = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        call("mg_kernel_info", self._h, ctypes.byref(r), ctypes.byref(t), ctypes.byref(l))
        return {"regs": r.value, "max_threads": t.value, "local_bytes": l.value}

    # ------------------------------------------------------------------ parameters
    def randomize(self, seed: int, lo: float = 0.8, hi: float = 1.2, current_sigma: float = 0.2,
                  nu0_sigma: float = 0.3, rg_halfwidth: float = 0.0, wait: bool = True):
        """Domain randomisation (mg_randomize).  wait=False returns without waiting
        (MG_RANDOMIZE_ASYNC: diagonal-mass fleets; a non-positive-definite mass matrix is then
        reported by sync())."""
        r = Ranges(lo, hi, current_sigma, nu0_sigma, 0 if wait else MG_RANDOMIZE_ASYNC,
                   rg_halfwidth)
        call("mg_randomize", self._h, ctypes.c_uint64(seed), ctypes.byref(r))

    def randomize_prefetch(self, seed: int, lo: float = 0.8, hi: float = 1.2,
                           current_sigma: float = 0.2):
        """Draw randomize(seed, lo, hi, current_sigma) ahead, on the library's own stream, into a
        second parameter buffer (mg_randomize_prefetch); the matching randomize() call installs
        it with one device copy.  Diagonal-mass fleets."""
        r = Ranges(lo, hi, current_sigma, 0.0, 0, 0.0)
        call("mg_randomize_prefetch", self._h, ctypes.c_uint64(seed), ctypes.byref(r))

    def set_params(self, params):
        _check(params, (self.n, MG_NPARAM), torch.float32)
        call("mg_set_params", self._h, _ptr(params))

    def get_params(self, out=None):
        if out is None:
            out = torch.empty((self.n, MG_NPARAM), dtype=torch.float32, device=self.device)
        _check(out, (self.n, MG_NPARAM), torch.float32)
        call("mg_get_params", self._h, _ptr(out))
        return out

    def set_hydro_offdiag(self, x):
        """Off-diagonal added mass and linear damping, float32 [n_envs, MG_NXPARAM] (layout of
        mg.h), or None for the diagonal model."""
        if x is None:
            call("mg_set_hydro_offdiag", self._h, None)
            return
        _check(x, (self.n, MG_NXPARAM), torch.float32)
        call("mg_set_hydro_offdiag", self._h, _ptr(x))

    def get_hydro_offdiag(self, out=None):
        if out is None:
            out = torch.empty((self.n, MG_NXPARAM), dtype=torch.float32, device=self.device)
        _check(out, (self.n, MG_NXPARAM), torch.float32)
        call("mg_get_hydro_offdiag", self._h, _ptr(out))
        return out

    # ------------------------------------------------------------------ actions and stepping
    def set_actions(self, actions, hold_steps: int = 1):
        """``actions``: float32 [n_seg, n_envs, w] (device tensor, or host tensor/array), w the
        action width (8 unless set_action_width(6))."""
        if actions is None:
            call("mg_set_actions", self._h, None, 0, int(hold_steps))
            return
        if actions.ndim != 3 or actions.shape[1:] != (self.n, self.act_w):
            raise ValueError(f"actions must be [n_seg, {self.n}, {self.act_w}]")
        _check(actions, actions.shape, torch.float32)
        call("mg_set_actions", self._h, _ptr(actions), int(actions.shape[0]), int(hold_steps))

    def set_actions_async(self, actions, hold_steps: int = 1):
        """As set_actions from a page-locked host tensor, without waiting (mg_set_actions_async):
        keep ``actions`` unchanged until ``sync()`` or the next-but-one call of this method."""
        if actions.ndim != 3 or actions.shape[1:] != (self.n, self.act_w):
            raise ValueError(f"actions must be [n_seg, {self.n}, {self.act_w}]")
        _check(actions, actions.shape, torch.float32)
        call("mg_set_actions_async", self._h, _ptr(actions), int(actions.shape[0]),
             int(hold_steps))

    def set_actions_borrowed(self, actions, hold_steps: int = 1):
        """Read ``actions`` (float32 device tensor [n_seg, n_envs, w]) in place, without a copy;
        keep it alive and unchanged until the steps using it have run (mg_set_actions_borrowed).
        """
        if not (isinstance(actions, torch.Tensor) and actions.is_cuda):
            raise ValueError("borrowed actions must be a CUDA tensor")
        if actions.ndim != 3 or actions.shape[1:] != (self.n, self.act_w):
            raise ValueError(f"actions must be [n_seg, {self.n}, {self.act_w}]")
        _check(actions, actions.shape, torch.float32)
        self._borrowed = actions  # keeps the storage alive while the sim may read it
        call("mg_set_actions_borrowed", self._h, _ptr(actions), int(actions.shape[0]),
             int(hold_steps))

    def set_action_width(self, width: int):
        """Floats per env and segment of later action buffers: 8 (default, zero-padded past a
        vehicle's thruster count) or 6 (fleets of 6-thruster vehicles; no padding).  Clears the
        current schedule (see mg_set_action_width)."""
        call("mg_set_action_width", self._h, int(width))
        self.act_w = int(width)

    def set_procedural_actions(self, cmd_seed: int, hold_steps: int):
        call("mg_set_procedural_actions", self._h, ctypes.c_uint64(cmd_seed), int(hold_steps))

    def step(self, k: int = 1):
        call("mg_step", self._h, int(k))

    def step_record(self, k: int, traj=None):
        """Advance k sub-steps writing the state after each to ``traj`` [k, 13, n] (device)."""
        if traj is None:
            traj = torch.empty((k, MG_NTRAJ, self.n), dtype=torch.float32, device=self.device)
        _check(traj, (k, MG_NTRAJ, self.n), torch.float32)
        call("mg_step_record", self._h, int(k), _ptr(traj))
        return traj

    def step_split(self, k: int, accel):
        """k sub-steps of the split-integration comparison scheme; ``accel`` [6, n] (device,
        float32) carries the previous sub-step's acceleration in and the last one out."""
        _check(accel, (6, self.n), torch.float32)
        call("mg_step_split", self._h, int(k), _ptr(accel))
        return accel

    # ------------------------------------------------------------------ task layer
    def set_task(self, task: int, centres, radius: float = 2.0, omega: float = 0.3,
                 vz: float = 0.1, psi_r: float = 0.0, lookahead: int = 4,
                 lookahead_dt: float = 0.5, max_error: float = 0.0, episode_steps: int = 0):
        """Task of §EXPERIMENTS (MG_TASK_*); centres: float32 [n, 4] (cx, cy, cz, phi0)."""
        spec = TaskSpec(int(task), int(lookahead), radius, omega, vz, psi_r, lookahead_dt,
                        max_error, int(episode_steps), 0)
        _check(centres, (self.n, 4), torch.float32)
        call("mg_set_task", self._h, ctypes.byref(spec), _ptr(centres))
        d = ctypes.c_int32()
        call("mg_task_obs_dim", self._h, ctypes.byref(d))
        self.obs_dim = d.value
        dev = self.device
        self._task_out = (torch.empty((self.n, self.obs_dim), dtype=torch.float32, device=dev),
                          torch.empty(self.n, dtype=torch.float32, device=dev),
                          torch.empty(self.n, dtype=torch.uint8, device=dev),
                          torch.empty(self.n, dtype=torch.float32, device=dev))
        self._task_ptrs = None

    def task_step(self, k: int):
        """(obs [n, obs_dim], err [n], done [n], episode_err [n]) after k sub-steps (k = 0:
        observe only).  The tensors are reused by the next call."""
        out = self._task_out
        if getattr(self, "_task_ptrs", None) is None or self._task_ptrs[0] is not out:
            # a policy loop calls this every few microseconds of GPU time: marshal the output
            # pointers once per set of buffers
            self._task_ptrs = (out, _lib.load(), tuple(_ptr(t) for t in out))
        _, lib, ptrs = self._task_ptrs
        st = lib.mg_task_step(self._h, int(k), *ptrs)
        if st != 0:
            raise MGError(st, "mg_task_step", lib.mg_last_error().decode(errors="replace"))
        return out

    # ------------------------------------------------------------------ state
    def get_state(self, out=None):
        if out is None:
            out = torch.empty((self.n, MG_NSTATE), dtype=torch.float32, device=self.device)
        _check(out, (self.n, MG_NSTATE), torch.float32)
        call("mg_get_state", self._h, _ptr(out))
        return out

    def get_state_async(self, out):
        """Read the state into a page-locked host tensor ``out`` [n, 21] without waiting
        (mg_get_state_async); ``out`` is complete once ``sync()`` returns."""
        _check(out, (self.n, MG_NSTATE), torch.float32)
        call("mg_get_state_async", self._h, _ptr(out))
        return out

    def set_state(self, state):
        _check(state, (self.n, MG_NSTATE), torch.float32)
        call("mg_set_state", self._h, _ptr(state))

    def reset(self, mask=None):
        if mask is None:
            call("mg_reset", self._h, None)
            return
        _check(mask, (self.n,), torch.uint8)
        call("mg_reset", self._h, _ptr(mask))

    def sync(self) -> int:
        """Wait for the stream; return how many envs are flagged non-finite."""
        c = ctypes.c_int64()
        call("mg_sync", self._h, ctypes.byref(c), ok=(0, 4))
        return c.value

    def nonfinite_mask(self):
        out = torch.empty(self.n, dtype=torch.uint8, device=self.device)
        call("mg_get_nonfinite", self._h, _ptr(out))
        return out

    # ------------------------------------------------------------------ lifetime
    def close(self):
        if self._h is not None:
            _lib.load().mg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def philox4x32_10(ctr, key) -> np.ndarray:
    """Evaluate Philox4x32-10 on the device for arrays ctr [n,4], key [n,2] (uint32)."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.zeros_like(ctr)
    call("mg_philox4x32_10", ctr.ctypes.data, key.ctypes.data, out.ctypes.data, ctr.shape[0])
    return out
