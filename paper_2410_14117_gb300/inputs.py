"""Seeded synthetic inputs for the Fossen fleet stepper.

This module is the one place that both the FP64 oracle tests and the CUDA path draw their inputs
from.  It holds vehicle definitions (the nominal BlueROV2 / BlueROV2-Heavy numbers and thruster
geometry of the experiments, §EXPERIMENTS) and seeded random draws (commands, states, per-env
parameter perturbations, fleet compositions, job arrivals).  It holds none of the equations of
motion: no rotation, no Coriolis, no damping, no integration.

Flat layouts used across the library boundary (documented again in ``include/mg.h``):

* parameters, ``NPARAM = 35`` per env::

      0 m | 1..3 Ixx Iyy Izz (about CG) | 4..9 added mass M_A diag | 10..15 linear damping diag
      16..21 quadratic damping diag | 22 W | 23 B | 24..26 r_g | 27..29 r_b | 30 k_T | 31 tau_m
      32..34 ocean current in NED

* state, ``NSTATE = 21`` per env: ``p(3) q(4: w,x,y,z) nu(6: u,v,w,p,q,r) n(8)`` — the lagged
  throttle ``n`` is zero past the vehicle's thruster count.

* thruster geometry per vehicle type: ``n_thr`` and positions ``r[8][3]``, unit directions
  ``d[8][3]`` in the body frame (x forward, y starboard, z down).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

NPARAM = 35
NXPARAM = 45  # off-diagonal extension: M_A above its diagonal (15), D_l off its diagonal (30)
NSTATE = 21
MAX_THR = 8
NCOEF = 18  # added-mass, linear-damping and quadratic-damping diagonals

P_M, P_IG, P_MA, P_DL, P_DQ = 0, 1, 4, 10, 16
P_W, P_B, P_RG, P_RB, P_KT, P_TAU, P_VC = 22, 23, 24, 27, 30, 31, 32
S_P, S_Q, S_NU, S_N = 0, 3, 7, 13

G_ACC = 9.81  # m/s^2; only used to derive the Heavy's weight from its mass

# The 27 scalars that domain randomisation scales by U[lo, hi] (§METHOD "physical parameter
# domain randomization"), in draw order.
RANDOMISED_INDICES = (
    [P_M, P_IG + 0, P_IG + 1, P_IG + 2]
    + [P_MA + i for i in range(6)]
    + [P_DL + i for i in range(6)]
    + [P_DQ + i for i in range(6)]
    + [P_W, P_B, P_RB + 2, P_KT, P_TAU]
)
assert len(RANDOMISED_INDICES) == 27

VEHICLE_BLUEROV2 = 0
VEHICLE_HEAVY = 1


@dataclasses.dataclass
class Vehicle:
    """Nominal parameters of one vehicle type (FP64) and its thruster geometry."""

    name: str
    params: np.ndarray  # float64 [NPARAM]
    n_thr: int
    r: np.ndarray  # float64 [MAX_THR, 3], zero past n_thr
    d: np.ndarray  # float64 [MAX_THR, 3], zero past n_thr

    def geo(self) -> np.ndarray:
        """Flat geometry record ``[n_thr, r(8x3), d(8x3)]`` (49 float64)."""
        return np.concatenate([[float(self.n_thr)], self.r.reshape(-1), self.d.reshape(-1)])


def _flu_to_frd(v):
    # The experiment's vectors are read as Isaac Sim's z-up / y-left body frame and converted to
    # the x-forward, y-starboard, z-down body frame the paper's NED convention implies.
    return (v[0], -v[1], -v[2])


def _base_params(m, frame):
    p = np.zeros(NPARAM)
    p[P_M] = m
    p[P_IG:P_IG + 3] = 0.16
    p[P_MA:P_MA + 6] = (5.5, 12.7, 14.57, 0.12, 0.12, 0.12)
    p[P_DL:P_DL + 6] = (4.03, 6.22, 5.18, 0.07, 0.07, 0.07)
    p[P_DQ:P_DQ + 6] = (18.18, 21.66, 36.99, 1.55, 1.55, 1.55)
    cb = (0.0, 0.0, 0.02)
    p[P_RB:P_RB + 3] = _flu_to_frd(cb) if frame == "stable" else cb
    p[P_RG:P_RG + 3] = 0.0
    p[P_KT] = 40.0
    p[P_TAU] = 0.05
    return p


def _horizontal(frame):
    s = 1.0 / math.sqrt(2.0)
    pos_cfg = [(0.156, 0.111, 0.085), (0.156, -0.111, 0.085),
               (-0.156, 0.111, 0.085), (-0.156, -0.111, 0.085)]
    if frame == "stable":
        pos = [_flu_to_frd(v) for v in pos_cfg]
    else:
        pos = pos_cfg
    # 45-degree vectored layout; direction chosen from the position's (x, y) quadrant in the
    # body frame: front thrusters point forward and inward-crossed, rear thrusters backward.
    dirs = []
    for (x, y, _z) in pos:
        if x > 0 and y > 0:
            dirs.append((s, -s, 0.0))
        elif x > 0:
            dirs.append((s, s, 0.0))
        elif y > 0:
            dirs.append((-s, -s, 0.0))
        else:
            dirs.append((-s, s, 0.0))
    return pos, dirs


def bluerov2(frame: str = "stable") -> Vehicle:
    """BlueROV2 (6 thrusters: 4 vectored horizontal, 2 vertical)."""
    p = _base_params(11.5, frame)
    p[P_W] = 112.8
    p[P_B] = 114.8
    pos, dirs = _horizontal(frame)
    for v in [(0.0, 0.111, 0.0), (0.0, -0.111, 0.0)]:
        pos.append(_flu_to_frd(v) if frame == "stable" else v)
        dirs.append((0.0, 0.0, 1.0))
    return _vehicle("BlueROV2", p, pos, dirs)


def bluerov2_heavy(frame: str = "stable") -> Vehicle:
    """BlueROV2 Heavy (8 thrusters: 4 vectored horizontal, 4 vertical).  Only the mass differs
    from the BlueROV2 in the experiment's numbers; the weight is m*g and the buoyancy keeps the
    BlueROV2's 2 N positive margin."""
    p = _base_params(13.5, frame)
    p[P_W] = 13.5 * G_ACC
    p[P_B] = 13.5 * G_ACC + 2.0
    pos, dirs = _horizontal(frame)
    for v in [(0.12, 0.218, 0.0), (0.12, -0.218, 0.0), (-0.12, 0.218, 0.0), (-0.12, -0.218, 0.0)]:
        pos.append(_flu_to_frd(v) if frame == "stable" else v)
        dirs.append((0.0, 0.0, 1.0))
    return _vehicle("BlueROV2-Heavy", p, pos, dirs)


def _vehicle(name, p, pos, dirs):
    r = np.zeros((MAX_THR, 3))
    d = np.zeros((MAX_THR, 3))
    r[:len(pos)] = np.array(pos, dtype=np.float64)
    d[:len(dirs)] = np.array(dirs, dtype=np.float64)
    r[r == 0.0] = 0.0  # no negative zeros
    return Vehicle(name=name, params=p, n_thr=len(pos), r=r, d=d)


def fleet_vehicles(frame: str = "stable"):
    """Vehicle table indexed by type id: 0 = BlueROV2, 1 = BlueROV2 Heavy."""
    return [bluerov2(frame), bluerov2_heavy(frame)]


def round_f32(x) -> np.ndarray:
    """Round to FP32 and promote back to FP64: both sides of a parity test read these values."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


# ----------------------------------------------------------------------------- random draws

def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def commands(seed: int, n_seg: int, n_envs: int, n_thr) -> np.ndarray:
    """Throttle commands c ~ U[-1, 1] per thruster and segment (Eq. 3 action space), float32
    ``[n_seg, n_envs, 8]``, zero past each env's thruster count.  ``n_thr`` is an int or a
    per-env array."""
    g = _rng(seed)
    c = g.uniform(-1.0, 1.0, size=(n_seg, n_envs, MAX_THR)).astype(np.float32)
    nt = np.broadcast_to(np.asarray(n_thr), (n_envs,))
    mask = np.arange(MAX_THR)[None, :] < nt[:, None]
    return c * mask[None, :, :]


def initial_states(seed: int, n_envs: int, nu_sigma: float = 0.3) -> np.ndarray:
    """Episode start: p = 0, identity attitude, body velocity nu ~ N(0, nu_sigma), throttle state
    n = 0.  float64 ``[n_envs, 21]``, every value already FP32-representable."""
    g = _rng(seed)
    s = np.zeros((n_envs, NSTATE))
    s[:, S_Q] = 1.0
    s[:, S_NU:S_NU + 6] = g.normal(0.0, nu_sigma, size=(n_envs, 6))
    return round_f32(s)


def random_states(seed: int, n_envs: int, n_thr, nu_sigma: float = 0.5,
                  pos_range: float = 5.0) -> np.ndarray:
    """Arbitrary states for single-step checks: uniform position, uniformly random unit
    attitude, normal body velocity, uniform throttle state in [-1, 1].  float64 ``[n, 21]``,
    FP32-representable; the attitude is unit to FP32 rounding."""
    g = _rng(seed)
    s = np.zeros((n_envs, NSTATE))
    s[:, S_P:S_P + 3] = g.uniform(-pos_range, pos_range, size=(n_envs, 3))
    q = g.normal(size=(n_envs, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1.0
    s[:, S_Q:S_Q + 4] = q
    s[:, S_NU:S_NU + 6] = g.normal(0.0, nu_sigma, size=(n_envs, 6))
    nt = np.broadcast_to(np.asarray(n_thr), (n_envs,))
    thr = g.uniform(-1.0, 1.0, size=(n_envs, MAX_THR))
    thr *= np.arange(MAX_THR)[None, :] < nt[:, None]
    s[:, S_N:S_N + MAX_THR] = thr
    return round_f32(s)


def perturbed_params(seed: int, nominal: np.ndarray, n_envs: int, lo: float = 0.8,
                     hi: float = 1.2, current_sigma: float = 0.2) -> np.ndarray:
    """Host-drawn per-env parameter sets: each randomised scalar times U[lo, hi], current
    ~ N(0, current_sigma) per NED axis.  ``nominal`` is ``[NPARAM]`` or ``[n_envs, NPARAM]``.
    float64 ``[n_envs, NPARAM]``, FP32-representable."""
    g = _rng(seed)
    p = np.array(np.broadcast_to(nominal, (n_envs, NPARAM)), dtype=np.float64)
    idx = np.array(RANDOMISED_INDICES)
    p[:, idx] *= g.uniform(lo, hi, size=(n_envs, idx.size))
    p[:, P_VC:P_VC + 3] += g.normal(0.0, current_sigma, size=(n_envs, 3))
    return round_f32(p)


def hydro_offdiag(seed: int, params: np.ndarray, coupling: float = 0.15) -> np.ndarray:
    """Off-diagonal added mass and linear damping for envs with records ``params`` [n, NPARAM]:
    M_A(i, j) = coupling * u * sqrt(M_A,ii M_A,jj) and D_l(i, j) = coupling * u' *
    sqrt(D_l,ii D_l,jj), u, u' ~ U[-1, 1] (D_l not symmetric), packed as the extension record
    (M_A above the diagonal row-major, then D_l off the diagonal row-major).  With coupling <
    0.2 every M_A stays diagonally dominant, so M_RB + M_A stays positive definite.  float64
    ``[n, NXPARAM]``, FP32-representable."""
    g = _rng(seed)
    n = params.shape[0]
    ma = params[:, P_MA:P_MA + 6]
    dl = params[:, P_DL:P_DL + 6]
    out = np.zeros((n, NXPARAM))
    t = 0
    for i in range(6):
        for j in range(i + 1, 6):
            out[:, t] = coupling * g.uniform(-1, 1, n) * np.sqrt(ma[:, i] * ma[:, j])
            t += 1
    for i in range(6):
        for j in range(6):
            if j != i:
                out[:, t] = coupling * g.uniform(-1, 1, n) * np.sqrt(dl[:, i] * dl[:, j])
                t += 1
    return round_f32(out)


def mixed_fleet(seed: int, total: int, max_group: int = 32768, p_first: float = 0.6) -> np.ndarray:
    """Mixed-fleet composition: groups with sizes log-uniform in [1, max_group] drawn until the
    sum reaches ``total`` (last group truncated); each group is BlueROV2 (type 0) with
    probability ``p_first``, else BlueROV2 Heavy (type 1).  int32 ``[total]`` of type ids."""
    g = _rng(seed)
    types = np.empty(total, dtype=np.int32)
    at = 0
    while at < total:
        size = int(math.floor(math.exp(g.uniform(0.0, math.log(max_group + 1.0)))))
        size = max(1, min(size, max_group, total - at))
        types[at:at + size] = 0 if g.uniform() < p_first else 1
        at += size
    return types


@dataclasses.dataclass
class JobSpec:
    arrival_s: float
    n_envs: int
    horizon: int
    vehicle: int
    param_seed: int
    cmd_seed: int


def serving_jobs(seed: int, duration_s: float, rate_hz: float = 200.0, env_lo: int = 64,
                 env_hi: int = 65536, h_lo: int = 50, h_hi: int = 1000) -> list:
    """Rollout-job stream: Poisson arrivals at ``rate_hz``; env count log-uniform in
    [env_lo, env_hi]; horizon uniform in [h_lo, h_hi] steps; vehicle type 50/50."""
    g = _rng(seed)
    jobs, t = [], 0.0
    while True:
        t += g.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        n = int(round(math.exp(g.uniform(math.log(env_lo), math.log(env_hi)))))
        jobs.append(JobSpec(arrival_s=t, n_envs=max(env_lo, min(env_hi, n)),
                            horizon=int(g.integers(h_lo, h_hi + 1)),
                            vehicle=int(g.integers(0, 2)),
                            param_seed=int(g.integers(1, 2**62)),
                            cmd_seed=int(g.integers(1, 2**62))))
    return jobs
