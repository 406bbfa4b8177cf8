"""Shared helpers of the parity tests: error metric, vehicle tables, oracle-side inputs."""
import numpy as np

from paper_2410_14117_gb300 import inputs as I

# Per-block error floors (p in m, q unitless, v in m/s, omega in rad/s, n unitless).
BLOCKS = [("p", I.S_P, 3, 1.0), ("q", I.S_Q, 4, 1.0), ("v", I.S_NU, 3, 0.1),
          ("w", I.S_NU + 3, 3, 0.1), ("n", I.S_N, 8, 1.0)]

TOL_STEP = 1e-5      # teacher-forced single sub-step
TOL_ROLLOUT = 1e-4   # after 500 sub-steps
TOL_QNORM = 1e-6     # | |q| - 1 | after every sub-step


def rel_err(gpu, ref):
    """Per env, per block b: |x_gpu - x_ref|_inf / max(|x_ref|_inf, floor_b); returns [n, 5]."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    out = np.zeros((ref.shape[0], len(BLOCKS)))
    for j, (_name, a, w, floor) in enumerate(BLOCKS):
        num = np.abs(gpu[:, a:a + w] - ref[:, a:a + w]).max(axis=1)
        den = np.maximum(np.abs(ref[:, a:a + w]).max(axis=1), floor)
        out[:, j] = num / den
    return out


def vehicles(frame="stable"):
    return I.fleet_vehicles(frame)


def oracle_geo(vs):
    """Oracle geometry records of the vehicles, FP32-rounded like the library's struct."""
    return np.stack([I.round_f32(v.geo()) for v in vs])


def oracle_nominal(vs):
    return np.stack([I.round_f32(v.params) for v in vs])


def f32(x):
    return float(np.float32(x))
