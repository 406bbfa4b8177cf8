"""Degenerate cases of Eq. 1 on the GPU, checked against what the mathematics fixes rather than
against the oracle: a neutral vehicle at rest stays exactly at rest, pure surge decays along the
closed form of linear + quadratic damping, and a pure yaw spin follows the closed-form
quaternion."""

import numpy as np
import pytest
import torch

from paper_2410_14117_gb300 import inputs as I
from paper_2410_14117_gb300.sim import Sim

from _helpers import oracle_nominal, vehicles

pytestmark = pytest.mark.gpu

def _neutral(p):
    p = p.copy()
    p[:, I.P_B] = p[:, I.P_W]
    p[:, I.P_RB:I.P_RB + 3] = p[:, I.P_RG:I.P_RG + 3]
    p[:, I.P_VC:I.P_VC + 3] = 0.0
    return p

def _sim(params, states, epb=128, spl=50, queue=False):
    vs = vehicles()
    n = params.shape[0]
    sim = Sim(n, np.zeros(n, np.int32), vs)
    sim.set_launch(epb, spl, True)
    sim.set_schedule(queue)
    sim.set_params(torch.tensor(params, dtype=torch.float32, device="cuda"))
    sim.set_state(torch.tensor(states, dtype=torch.float32, device="cuda"))
    sim.set_actions(None, 1)  # zero commands
    return sim

@pytest.mark.parametrize("queue", [False, True])
def test_neutral_vehicle_at_rest_stays_exactly_at_rest(queue):
    """W = B, r_b = r_g, no current, nu = 0, n = 0, c = 0: every term of Eq. 1 is an exact zero,
    so p, nu and n keep their bits; q only meets the renormalisation (within 2 ulp)."""
    vs = vehicles()
    n = 2048
    params = _neutral(I.perturbed_params(1, oracle_nominal(vs)[[0]], n))
    states = I.random_states(2, n, 6)
    states[:, I.S_NU:] = 0.0
    sim = _sim(params, states, queue=queue)
    sim.step(300)
    got = sim.get_state().cpu().numpy()
    sim.close()
    want = states.astype(np.float32)
    np.testing.assert_array_equal(got[:, I.S_P:I.S_P + 3], want[:, I.S_P:I.S_P + 3])
    np.testing.assert_array_equal(got[:, I.S_NU:], want[:, I.S_NU:])
    np.testing.assert_allclose(got[:, I.S_Q:I.S_Q + 4], want[:, I.S_Q:I.S_Q + 4], rtol=0,
                               atol=2.5e-7)

def test_pure_surge_decay_closed_form():
    """Neutral, no current, surge only: (m + M_A,u) u' = -(d_l + d_q |u|) u, whose solution is
    u(t) = a u0 e^{-a t/m'} / (a + b u0 (1 - e^{-a t/m'})) with a = d_l, b = d_q, m' = m + M_A,u.
    Nominal BlueROV2 from u0 = 0.3 m/s: u(1 s) = 0.184099, u(5 s) = 0.047274."""
    vs = vehicles()
    n = 64
    params = _neutral(np.repeat(oracle_nominal(vs)[[0]], n, axis=0))
    u0 = np.linspace(0.05, 0.6, n)
    states = np.zeros((n, I.NSTATE))
    states[:, I.S_Q] = 1.0
    states[:, I.S_NU] = I.round_f32(u0)
    sim = _sim(params, states)
    a, b = params[0, I.P_DL], params[0, I.P_DQ]
    mp = params[0, I.P_M] + params[0, I.P_MA]
    t = 0.0
    for steps in (100, 400):
        sim.step(steps)
        t += steps * 0.01
        got = sim.get_state().double().cpu().numpy()
        x = np.exp(-a * t / mp)
        u = a * states[:, I.S_NU] * x / (a + b * states[:, I.S_NU] * (1 - x))
        np.testing.assert_allclose(got[:, I.S_NU], u, rtol=2e-5, atol=1e-8)
        # the surge distance is the integral of u: m'/b ln(1 + b u0 (1 - x) / a)
        dist = mp / b * np.log1p(b * states[:, I.S_NU] * (1 - x) / a)
        np.testing.assert_allclose(got[:, I.S_P], dist, rtol=2e-5, atol=1e-7)
        assert np.abs(got[:, I.S_NU + 1:I.S_NU + 6]).max() == 0.0
    sim.close()
    i = int(np.argmin(np.abs(u0 - 0.3)))
    assert abs(u0[i] - 0.3) < 0.005

def test_pure_surge_reference_values():
    vs = vehicles()
    params = _neutral(oracle_nominal(vs)[[0]])
    states = np.zeros((1, I.NSTATE))
    states[0, I.S_Q] = 1.0
    states[0, I.S_NU] = 0.3
    sim = _sim(params, states)
    sim.step(100)
    u1 = float(sim.get_state()[0, I.S_NU])
    sim.step(400)
    u5 = float(sim.get_state()[0, I.S_NU])
    sim.close()
    assert abs(u1 - 0.184099) < 2e-6 and abs(u5 - 0.047274) < 2e-6

def test_pure_yaw_spin_closed_form_quaternion():
    """Undamped, neutral, isotropic inertia, yaw rate r: the spin is steady and
    q(t) = (cos(r t/2), 0, 0, sin(r t/2)); the heading after 2 s must match to FP32 rounding."""
    vs = vehicles()
    n = 32
    params = _neutral(np.repeat(oracle_nominal(vs)[[0]], n, axis=0))
    params[:, I.P_DL:I.P_DQ + 6] = 0.0
    params[:, I.P_IG:I.P_IG + 3] = 0.16
    params[:, I.P_MA + 3:I.P_MA + 6] = 0.12
    r = np.linspace(-2.0, 2.0, n)
    states = np.zeros((n, I.NSTATE))
    states[:, I.S_Q] = 1.0
    states[:, I.S_NU + 5] = I.round_f32(r)
    sim = _sim(params, states)
    sim.step(200)
    got = sim.get_state().double().cpu().numpy()
    sim.close()
    th = states[:, I.S_NU + 5] * 2.0 / 2
    want = np.stack([np.cos(th), np.zeros(n), np.zeros(n), np.sin(th)], axis=1)
    np.testing.assert_allclose(got[:, I.S_Q:I.S_Q + 4], want, rtol=0, atol=1e-5)
    np.testing.assert_allclose(got[:, I.S_NU + 5], states[:, I.S_NU + 5], rtol=0, atol=0)
