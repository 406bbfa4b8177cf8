"""ctypes wrapper of the FP64 CPU oracle (``fossen_oracle.c``) — TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg import this
module.  It never imports the CUDA package and the CUDA package never imports it.

Every function follows Eq. 1 of §METHOD (the extended Fossen equation), with the readings stated
in the C file's header.  Arrays are float64, C-contiguous.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

NPARAM = 35
NSTATE = 21
NGEO = 49
MAX_THR = 8
NO_CURRENT_ACCEL = 1
NXPARAM = 45        # off-diagonal extension: M_A above the diagonal (15), D_l off-diagonal (30)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fossen_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_I32 = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available).  FP contraction is off so that the
    x86 and Arm builds round identically."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o",
            _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_rotation.argtypes = [_D, _D]
            for name in ("orc_mass_rb", "orc_mass_a"):
                getattr(L, name).argtypes = [_D, _D]
            for name in ("orc_coriolis_rb", "orc_coriolis_a", "orc_damping", "orc_restoring"):
                getattr(L, name).argtypes = [_D, _D, _D]
            L.orc_thrust.argtypes = [_D, _D, _D, _D]
            L.orc_rhs.argtypes = [_D, _D, _D, _D, ctypes.c_int, _D]
            L.orc_rhs.restype = ctypes.c_int
            L.orc_rk4_step.argtypes = [_D, _D, _D, _D, ctypes.c_double, ctypes.c_int, _D]
            L.orc_rk4_step.restype = ctypes.c_int
            L.orc_rollout.argtypes = [ctypes.c_int64, _D, _D, _I32, _D, _D, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                      ctypes.c_int32, _D, ctypes.c_int32]
            L.orc_rollout.restype = ctypes.c_int64
            L.orc_max_threads.restype = ctypes.c_int
            L.orc_philox4x32_10.argtypes = [_U32, _U32, _U32]
            L.orc_randomize.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double, _D,
                                        _I32, ctypes.c_int64, _D]
            L.orc_mass_a_x.argtypes = [_D, _D, _D]
            L.orc_coriolis_a_x.argtypes = [_D, _D, _D, _D]
            L.orc_damping_x.argtypes = [_D, _D, _D, _D]
            L.orc_rhs_x.argtypes = [_D, _D, _D, _D, _D, ctypes.c_int, _D]
            L.orc_rhs_x.restype = ctypes.c_int
            L.orc_rollout_x.argtypes = [ctypes.c_int64, _D, _D, _D, _I32, _D, _D, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                        ctypes.c_int32, _D, ctypes.c_int32]
            L.orc_rollout_x.restype = ctypes.c_int64
            L.orc_reset_state.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_int64,
                                          ctypes.c_uint32, _D]
            L.orc_commands.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32,
                                       ctypes.c_int32, _D]
            L.orc_euler_zyx.argtypes = [_D, _D]
            L.orc_task_reference.argtypes = [ctypes.c_int32, _D, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double, _D]
            L.orc_task_observe.argtypes = [ctypes.c_int32, _D, _D, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int32, ctypes.c_double, ctypes.c_double, _D]
            L.orc_task_observe.restype = ctypes.c_double
            L.orc_split_step_x.argtypes = [_D, _D, _D, _D, _D, _D, ctypes.c_double,
                                           ctypes.c_int, _D, _D]
            L.orc_split_step_x.restype = ctypes.c_int
            L.orc_split_rollout_x.argtypes = [ctypes.c_int64, _D, _D, _D, _I32, _D, _D, _D,
                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_double, ctypes.c_int32, ctypes.c_int32]
            L.orc_split_rollout_x.restype = ctypes.c_int64
            _lib = L
    return _lib


def _p(a, ct=_D):
    return a.ctypes.data_as(ct)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# ------------------------------------------------------------------ single-env model terms

def rotation(q) -> np.ndarray:
    q = _f64(q, (4,))
    R = np.zeros(9)
    lib().orc_rotation(_p(q), _p(R))
    return R.reshape(3, 3)


def _mat(fn, par, *vecs):
    par = _f64(par, (NPARAM,))
    out = np.zeros(36)
    args = [_p(par)] + [_p(_f64(v)) for v in vecs] + [_p(out)]
    getattr(lib(), fn)(*args)
    return out.reshape(6, 6)


def mass_rb(par):
    return _mat("orc_mass_rb", par)


def mass_a(par, xpar=None):
    if xpar is None:
        return _mat("orc_mass_a", par)
    out = np.zeros(36)
    lib().orc_mass_a_x(_p(_f64(par, (NPARAM,))), _p(_f64(xpar, (NXPARAM,))), _p(out))
    return out.reshape(6, 6)


def coriolis_rb(par, nu):
    return _mat("orc_coriolis_rb", par, nu)


def coriolis_a(par, nu_r, xpar=None):
    if xpar is None:
        return _mat("orc_coriolis_a", par, nu_r)
    out = np.zeros(36)
    lib().orc_coriolis_a_x(_p(_f64(par, (NPARAM,))), _p(_f64(xpar, (NXPARAM,))),
                           _p(_f64(nu_r, (6,))), _p(out))
    return out.reshape(6, 6)


def damping(par, nu_r, xpar=None):
    if xpar is None:
        return _mat("orc_damping", par, nu_r)
    out = np.zeros(36)
    lib().orc_damping_x(_p(_f64(par, (NPARAM,))), _p(_f64(xpar, (NXPARAM,))),
                        _p(_f64(nu_r, (6,))), _p(out))
    return out.reshape(6, 6)


def restoring(par, q) -> np.ndarray:
    par = _f64(par, (NPARAM,))
    g = np.zeros(6)
    lib().orc_restoring(_p(par), _p(_f64(q, (4,))), _p(g))
    return g


def thrust(par, geo, n) -> np.ndarray:
    tau = np.zeros(6)
    n8 = np.zeros(MAX_THR)
    n = np.asarray(n, dtype=np.float64)
    n8[:n.size] = n
    lib().orc_thrust(_p(_f64(par, (NPARAM,))), _p(_f64(geo, (NGEO,))), _p(n8), _p(tau))
    return tau


def rhs(par, geo, s, c, flags: int = 0, xpar=None) -> np.ndarray:
    ds = np.zeros(NSTATE)
    c8 = np.zeros(MAX_THR)
    c = np.asarray(c, dtype=np.float64)
    c8[:c.size] = c
    xp = None if xpar is None else _p(_f64(xpar, (NXPARAM,)))
    rc = lib().orc_rhs_x(_p(_f64(par, (NPARAM,))), xp, _p(_f64(geo, (NGEO,))),
                         _p(_f64(s, (NSTATE,))), _p(c8), flags, _p(ds))
    if rc != 0:
        raise FloatingPointError("singular mass matrix")
    return ds


def rk4_step(par, geo, s, c, h: float, flags: int = 0) -> np.ndarray:
    out = np.zeros(NSTATE)
    c8 = np.zeros(MAX_THR)
    c = np.asarray(c, dtype=np.float64)
    c8[:c.size] = c
    rc = lib().orc_rk4_step(_p(_f64(par, (NPARAM,))), _p(_f64(geo, (NGEO,))),
                            _p(_f64(s, (NSTATE,))), _p(c8), h, flags, _p(out))
    if rc != 0:
        raise FloatingPointError("singular mass matrix")
    return out


# ------------------------------------------------------------------ fleet rollout

def rollout(par, geo, types, s0, cmd, hold: int, n_steps: int, h: float = 0.01,
            flags: int = 0, record: bool = False, nthreads: int = 0, xpar=None):
    """Advance every env ``n_steps`` RK4 steps.

    par [n, NPARAM]; geo [n_types, NGEO]; types int [n]; s0 [n, NSTATE]; cmd [n_seg, n, 8] with
    step j using segment min(j // hold, n_seg - 1).  Returns the final state [n, NSTATE] and,
    with ``record``, the trajectory [n_steps, n, NSTATE] (state after every step)."""
    par = _f64(par)
    n = par.shape[0]
    geo = _f64(geo).reshape(-1, NGEO)
    types = np.ascontiguousarray(types, dtype=np.int32).reshape(n)
    s = _f64(s0).reshape(n, NSTATE).copy()
    cmd = _f64(cmd).reshape(-1, n, MAX_THR)
    traj = np.zeros((n_steps, n, NSTATE)) if record else None
    xp = None if xpar is None else _f64(xpar).reshape(n, NXPARAM)
    fails = lib().orc_rollout_x(n, _p(par), _p(xp) if xp is not None else None, _p(geo),
                                _p(types, _I32), _p(s), _p(cmd), cmd.shape[0], hold, n_steps, h,
                                flags, _p(traj) if record else None, nthreads)
    if fails:
        raise FloatingPointError(f"{fails} envs had a singular mass matrix")
    return (s, traj) if record else s


def max_threads() -> int:
    return lib().orc_max_threads()


# ------------------------------------------------------------------ counter-based draws

def philox4x32_10(ctr, key) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(ctr, _U32), _p(key, _U32), _p(out, _U32))
    return out


def randomize(seed: int, nominal, types, lo: float = 0.8, hi: float = 1.2,
              current_sigma: float = 0.2, gid0: int = 0, rg_halfwidth: float = 0.0) -> np.ndarray:
    """Per-env domain-randomised parameters [n, NPARAM] (FP64)."""
    nominal = _f64(nominal).reshape(-1, NPARAM)
    types = np.ascontiguousarray(types, dtype=np.int32)
    out = np.zeros((types.size, NPARAM))
    lib().orc_randomize(types.size, seed, lo, hi, current_sigma, rg_halfwidth, _p(nominal),
                        _p(types, _I32), gid0, _p(out))
    return out


def reset_state(seed: int, nu0_sigma: float, gid: int, episode: int) -> np.ndarray:
    s = np.zeros(NSTATE)
    lib().orc_reset_state(seed, nu0_sigma, gid, episode, _p(s))
    return s


def commands(cmd_seed: int, gid: int, seg: int, n_thr: int) -> np.ndarray:
    c = np.zeros(MAX_THR)
    lib().orc_commands(cmd_seed, gid, seg, n_thr, _p(c))
    return c


# ------------------------------------------------------------------ task layer (§EXPERIMENTS)

TASK_STATION, TASK_CIRCLE, TASK_HELIX, TASK_LEMNISCATE = 0, 1, 2, 3


def euler_zyx(q) -> np.ndarray:
    e = np.zeros(3)
    lib().orc_euler_zyx(_p(_f64(q, (4,))), _p(e))
    return e


def task_reference(task: int, centre, radius: float, omega: float, vz: float, t: float):
    p = np.zeros(3)
    lib().orc_task_reference(task, _p(_f64(centre, (4,))), radius, omega, vz, t, _p(p))
    return p


def task_observe(task: int, s, centre, radius, omega, vz, psi_r, m, dt_look, t):
    """(obs [6 m' + 6], position error) of one env (Eq. 2, Eq. 4); m' = 1 for station keeping."""
    mm = 1 if task == TASK_STATION else m
    obs = np.zeros(6 * mm + 6)
    err = lib().orc_task_observe(task, _p(_f64(s, (NSTATE,))), _p(_f64(centre, (4,))), radius,
                                 omega, vz, psi_r, m, dt_look, t, _p(obs))
    return obs, err


# ------------------------------------------------------------------ split integration (§METHOD)

def split_step(par, geo, s, a, c, h: float, flags: int = 0, xpar=None):
    """One sub-step of the split scheme (rigid body by semi-implicit Euler, hydrodynamic term as
    an external force with the previous acceleration ``a`` in its added-mass part); xpar: the
    off-diagonal extension of M_A and D_l, or None.  Returns (state, acceleration)."""
    out = np.zeros(NSTATE)
    a_out = np.zeros(6)
    c8 = np.zeros(MAX_THR)
    c = np.asarray(c, dtype=np.float64)
    c8[:c.size] = c
    xp = None if xpar is None else _p(_f64(xpar, (NXPARAM,)))
    rc = lib().orc_split_step_x(_p(_f64(par, (NPARAM,))), xp, _p(_f64(geo, (NGEO,))),
                                _p(_f64(s, (NSTATE,))), _p(_f64(a, (6,))), _p(c8), h, flags,
                                _p(out), _p(a_out))
    if rc != 0:
        raise FloatingPointError("singular rigid-body mass matrix")
    return out, a_out


def split_rollout(par, geo, types, s0, a0, cmd, hold: int, n_steps: int, h: float = 0.01,
                  flags: int = 0, nthreads: int = 0, xpar=None):
    """Fleet rollout of the split scheme; returns (state [n, NSTATE], acceleration [n, 6])."""
    par = _f64(par)
    n = par.shape[0]
    geo = _f64(geo).reshape(-1, NGEO)
    types = np.ascontiguousarray(types, dtype=np.int32).reshape(n)
    s = _f64(s0).reshape(n, NSTATE).copy()
    a = _f64(a0).reshape(n, 6).copy()
    cmd = _f64(cmd).reshape(-1, n, MAX_THR)
    xp = None if xpar is None else _f64(xpar).reshape(n, NXPARAM)
    fails = lib().orc_split_rollout_x(n, _p(par), _p(xp) if xp is not None else None, _p(geo),
                                      _p(types, _I32), _p(s), _p(a), _p(cmd), cmd.shape[0], hold,
                                      n_steps, h, flags, nthreads)
    if fails:
        raise FloatingPointError(f"{fails} envs had a singular rigid-body mass matrix")
    return s, a
