"""ctypes binding of libmg.so (the C ABI in include/mg.h).  Argument marshalling only.

The library is built in-tree on first use if it is missing or stale; if it cannot be built or
loaded, every call raises — there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import threading

from . import build as _build

MG_NPARAM = 35
MG_NXPARAM = 45
MG_RANDOMIZE_ASYNC = 1
MG_NSTATE = 21
MG_NTRAJ = 13
MG_MAX_THR = 8
MG_MAX_TYPES = 8
MG_MODEL_NO_CURRENT_ACCEL = 1
MG_TASK_STATION, MG_TASK_CIRCLE, MG_TASK_HELIX, MG_TASK_LEMNISCATE = 0, 1, 2, 3

STATUS = {0: "MG_OK", 1: "MG_EINVAL", 2: "MG_ENOMEM", 3: "MG_ECUDA", 4: "MG_ENONFINITE",
          5: "MG_ENOTSPD", 6: "MG_ETIMEOUT", 7: "MG_ESTATE"}


class MGError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        self.code = STATUS.get(status, str(status))
        super().__init__(f"{where}: {self.code}: {message}")


class VehicleParams(ctypes.Structure):
    _fields_ = [("m", ctypes.c_float), ("Ixx", ctypes.c_float), ("Iyy", ctypes.c_float),
                ("Izz", ctypes.c_float), ("MA", ctypes.c_float * 6), ("Dl", ctypes.c_float * 6),
                ("Dq", ctypes.c_float * 6), ("W", ctypes.c_float), ("B", ctypes.c_float),
                ("rg", ctypes.c_float * 3), ("rb", ctypes.c_float * 3), ("kT", ctypes.c_float),
                ("tau_m", ctypes.c_float), ("n_thr", ctypes.c_int32),
                ("r", (ctypes.c_float * 3) * MG_MAX_THR),
                ("d", (ctypes.c_float * 3) * MG_MAX_THR)]


class Ranges(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float), ("hi", ctypes.c_float),
                ("current_sigma", ctypes.c_float), ("nu0_sigma", ctypes.c_float),
                ("flags", ctypes.c_uint32), ("rg_halfwidth", ctypes.c_float)]


class TaskSpec(ctypes.Structure):
    _fields_ = [("task", ctypes.c_int32), ("lookahead", ctypes.c_int32),
                ("radius", ctypes.c_float), ("omega", ctypes.c_float), ("vz", ctypes.c_float),
                ("psi_r", ctypes.c_float), ("lookahead_dt", ctypes.c_float),
                ("max_error", ctypes.c_float), ("episode_steps", ctypes.c_int32),
                ("flags", ctypes.c_uint32)]


class JobSpec(ctypes.Structure):
    _fields_ = [("n_envs", ctypes.c_int64), ("vehicle_type", ctypes.c_int32),
                ("hold_steps", ctypes.c_int32), ("horizon", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("param_seed", ctypes.c_uint64),
                ("cmd_seed", ctypes.c_uint64), ("ranges", Ranges)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_double), ("k", ctypes.c_int32),
                ("max_inflight", ctypes.c_int32), ("record", ctypes.c_int32),
                ("serial", ctypes.c_int32), ("keep_done", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("wait_timeout_s", ctypes.c_double)]


_P = ctypes.c_void_p
_I32, _I64, _U32, _U64, _F = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64,
                              ctypes.c_float)
_D = ctypes.c_double

# name -> argtypes (every entry point returns mg_status except mg_last_error)
SIGNATURES = {
    "mg_create": [_I64, _P, ctypes.POINTER(VehicleParams), _I32, ctypes.POINTER(_P)],
    "mg_destroy": [_P],
    "mg_set_stream": [_P, _P],
    "mg_set_env_id_offset": [_P, _I64],
    "mg_set_model_flags": [_P, _U32],
    "mg_set_timestep": [_P, _F],
    "mg_set_launch": [_P, _I32, _I32, _I32],
    "mg_set_schedule": [_P, _I32, _I32, _I32],
    "mg_set_wait_limit": [_P, ctypes.c_uint32],
    "mg_randomize": [_P, _U64, ctypes.POINTER(Ranges)],
    "mg_randomize_prefetch": [_P, _U64, ctypes.POINTER(Ranges)],
    "mg_set_adjoint_mode": [_P, _I32],
    "mg_set_params": [_P, _P],
    "mg_get_params": [_P, _P],
    "mg_set_actions": [_P, _P, _I32, _I32],
    "mg_set_actions_borrowed": [_P, _P, _I32, _I32],
    "mg_set_actions_async": [_P, _P, _I32, _I32],
    "mg_set_action_width": [_P, _I32],
    "mg_get_state_async": [_P, _P],
    "mg_set_procedural_actions": [_P, _U64, _I32],
    "mg_step": [_P, _I32],
    "mg_step_noalloc": [_P, _I32],
    "mg_step_record": [_P, _I32, _P],
    "mg_step_split": [_P, _I32, _P],
    "mg_set_hydro_offdiag": [_P, _P],
    "mg_get_hydro_offdiag": [_P, _P],
    "mg_rollout_forward": [_P, _I32, _I32, _P, _P, ctypes.POINTER(_I64)],
    "mg_rollout_backward": [_P, _I32, _I32, _P, _P, _I64, _P, _P, _P],
    "mg_get_state": [_P, _P],
    "mg_set_state": [_P, _P],
    "mg_reset": [_P, _P],
    "mg_sync": [_P, ctypes.POINTER(_I64)],
    "mg_get_nonfinite": [_P, _P],
    "mg_philox4x32_10": [_P, _P, _P, _I64],
    "mg_kernel_info": [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32)],
    "mg_set_task": [_P, ctypes.POINTER(TaskSpec), _P],
    "mg_task_obs_dim": [_P, ctypes.POINTER(_I32)],
    "mg_task_step": [_P, _I32, _P, _P, _P, _P],
    "mg_env_step": [_P, _I32, _P, _P, _P, _P, _P],
    "mg_pool_create": [_I64, ctypes.POINTER(VehicleParams), _I32, ctypes.POINTER(_P)],
    "mg_pool_destroy": [_P],
    "mg_pool_set_stream": [_P, _P],
    "mg_pool_admit": [_P, ctypes.POINTER(JobSpec), _P, ctypes.POINTER(_I32)],
    "mg_pool_admit_offdiag": [_P, ctypes.POINTER(JobSpec), _P, _P, ctypes.POINTER(_I32)],
    "mg_server_submit_offdiag": [_P, ctypes.POINTER(JobSpec), _P, ctypes.POINTER(_I64)],
    "mg_pool_tick": [_P, _I32, ctypes.POINTER(_I32)],
    "mg_pool_job_progress": [_P, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32)],
    "mg_pool_get_job_state": [_P, _I32, _P],
    "mg_pool_release": [_P, _I32],
    "mg_pool_info": [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I32)],
    "mg_pool_sync": [_P],
    "mg_server_create": [_P, ctypes.POINTER(ServerConfig), ctypes.POINTER(_P)],
    "mg_server_destroy": [_P],
    "mg_server_submit": [_P, ctypes.POINTER(JobSpec), ctypes.POINTER(_I64)],
    "mg_server_poll": [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32)],
    "mg_server_job": [_P, _I64, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_D)],
    "mg_server_job_result": [_P, _I64, _P, _P],
    "mg_server_release": [_P, _I64],
    "mg_server_info": [_P, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_D)],
}

_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    """Build (if needed) and load libmg.so, declaring every entry point's signature."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)
            for name, args in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            L.mg_last_error.argtypes = []
            L.mg_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def call(name: str, *args, ok=(0,)) -> int:
    """Call an entry point; raise MGError unless its status is in ``ok``."""
    L = load()
    st = getattr(L, name)(*args)
    if st not in ok:
        raise MGError(st, name, L.mg_last_error().decode(errors="replace"))
    return st
