"""Pins of the FP64 oracle against facts fixed by the paper's model and by the mathematics.

Each check is chosen so that a plausible slip in the oracle (a dropped term, a flipped sign, a
transposed rotation, a wrong RK4 weight) fails it.  None of these checks re-types the oracle's
own formulas: they use textbook closed forms (Euler-angle restoring vector and rotation,
Newton-Euler rigid-body equations, exact solutions of 1-D problems), conservation laws and
brute force.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_14117_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


# ----------------------------------------------------------------------------- helpers

def quat_from_euler(phi, theta, psi):
    """zyx (yaw-pitch-roll) Euler angles -> unit quaternion (w, x, y, z)."""
    cp, sp = math.cos(phi / 2), math.sin(phi / 2)
    ct, st = math.cos(theta / 2), math.sin(theta / 2)
    cs, ss = math.cos(psi / 2), math.sin(psi / 2)
    return np.array([cp * ct * cs + sp * st * ss, sp * ct * cs - cp * st * ss,
                     cp * st * cs + sp * ct * ss, cp * ct * ss - sp * st * cs])


def rot_euler(phi, theta, psi):
    """Body -> NED rotation Rz(psi) Ry(theta) Rx(phi)."""
    cx, sx = math.cos(phi), math.sin(phi)
    cy, sy = math.cos(theta), math.sin(theta)
    cz, sz = math.cos(psi), math.sin(psi)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def restoring_euler(par, phi, theta):
    """Fossen's Euler-angle closed form of g(eta) for weight W at r_g, buoyancy B at r_b."""
    W, B = par[I.P_W], par[I.P_B]
    xg, yg, zg = par[I.P_RG:I.P_RG + 3]
    xb, yb, zb = par[I.P_RB:I.P_RB + 3]
    s_th, c_th, s_ph, c_ph = math.sin(theta), math.cos(theta), math.sin(phi), math.cos(phi)
    return np.array([
        (W - B) * s_th,
        -(W - B) * c_th * s_ph,
        -(W - B) * c_th * c_ph,
        -(yg * W - yb * B) * c_th * c_ph + (zg * W - zb * B) * c_th * s_ph,
        (zg * W - zb * B) * s_th + (xg * W - xb * B) * c_th * c_ph,
        -(xg * W - xb * B) * c_th * s_ph - (yg * W - yb * B) * s_th,
    ])


def state(p=(0, 0, 0), q=(1, 0, 0, 0), nu=(0,) * 6, n=()):
    s = np.zeros(I.NSTATE)
    s[I.S_P:I.S_P + 3] = p
    s[I.S_Q:I.S_Q + 4] = q
    s[I.S_NU:I.S_NU + 6] = nu
    s[I.S_N:I.S_N + len(n)] = n
    return s


def neutral(par):
    """Neutrally buoyant, CB at CG, no current: no restoring force, no current terms."""
    p = par.copy()
    p[I.P_B] = p[I.P_W]
    p[I.P_RB:I.P_RB + 3] = p[I.P_RG:I.P_RG + 3]
    p[I.P_VC:I.P_VC + 3] = 0.0
    return p


def undamped(par):
    p = par.copy()
    p[I.P_DL:I.P_DL + 6] = 0.0
    p[I.P_DQ:I.P_DQ + 6] = 0.0
    return p


def one_thruster_vehicle(r=(0, 0, 0), d=(1, 0, 0)):
    geo = np.zeros(O.NGEO)
    geo[0] = 1
    geo[1:4] = r
    geo[1 + 3 * O.MAX_THR:4 + 3 * O.MAX_THR] = d
    return geo


def rollout1(par, geo, s0, c, n_steps, h=0.01, flags=0, xpar=None):
    cmd = np.zeros((1, 1, 8))
    cmd[0, 0, :len(c)] = c
    s, traj = O.rollout(par[None], geo[None], [0], s0[None], cmd, 1, n_steps, h=h, flags=flags,
                        record=True, xpar=None if xpar is None else xpar[None])
    return s[0], traj[:, 0]


V = I.bluerov2()
VH = I.bluerov2_heavy()
GEO = V.geo()


# ----------------------------------------------------------------------------- counter RNG

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


# ----------------------------------------------------------------------------- attitude

def test_rotation_matches_euler_angles():
    g = np.random.default_rng(3)
    for _ in range(50):
        phi, theta, psi = g.uniform(-math.pi, math.pi), g.uniform(-1.5, 1.5), g.uniform(-3, 3)
        R = O.rotation(quat_from_euler(phi, theta, psi))
        np.testing.assert_allclose(R, rot_euler(phi, theta, psi), atol=1e-14)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)


# ----------------------------------------------------------------------------- restoring

def test_restoring_golden_values():
    rows = [list(map(float, l.split())) for l in
            open(os.path.join(HERE, "golden", "restoring_closed_form.txt"))
            if l.strip() and not l.startswith("#")]
    for r in rows:
        q = quat_from_euler(math.radians(r[0]), math.radians(r[1]), 0.0)
        np.testing.assert_allclose(O.restoring(V.params, q), r[2:], atol=5e-7)


@pytest.mark.parametrize("frame", ["stable", "literal"])
def test_restoring_matches_euler_closed_form(frame):
    par = I.bluerov2(frame).params.copy()
    g = np.random.default_rng(4)
    for k in range(40):
        p = par.copy()
        if k % 2:  # off-centre gravity as well
            p[I.P_RG:I.P_RG + 3] = g.uniform(-0.05, 0.05, 3)
            p[I.P_RB:I.P_RB + 3] = g.uniform(-0.05, 0.05, 3)
        phi, theta, psi = g.uniform(-3, 3), g.uniform(-1.5, 1.5), g.uniform(-3, 3)
        np.testing.assert_allclose(O.restoring(p, quat_from_euler(phi, theta, psi)),
                                   restoring_euler(p, phi, theta), atol=1e-12)


def test_literal_frame_flips_righting_moment():
    q = quat_from_euler(math.radians(20), 0, 0)
    gs = O.restoring(I.bluerov2("stable").params, q)
    gl = O.restoring(I.bluerov2("literal").params, q)
    assert gs[3] > 0 and gl[3] < 0  # stable: -g pushes back; literal: pushes further over
    np.testing.assert_allclose(gs[3], -gl[3], rtol=1e-12)


# ----------------------------------------------------------------------------- inertia

def test_mass_matrix_nominal_and_spd():
    M = O.mass_rb(V.params) + O.mass_a(V.params)
    np.testing.assert_allclose(M, np.diag([17.0, 24.2, 26.07, 0.28, 0.28, 0.28]), atol=1e-12)
    g = np.random.default_rng(5)
    for _ in range(50):
        p = I.perturbed_params(int(g.integers(1 << 30)), V.params, 1)[0]
        p[I.P_RG:I.P_RG + 3] = g.uniform(-0.05, 0.05, 3)
        M = O.mass_rb(p) + O.mass_a(p)
        np.testing.assert_allclose(M, M.T, atol=1e-15)
        assert np.linalg.eigvalsh(M).min() > 0
        np.testing.assert_allclose(M @ np.linalg.inv(M), np.eye(6), atol=1e-13)


def test_rigid_body_kinetic_energy_parallel_axis():
    """1/2 nu^T M_RB nu equals the CG form 1/2 m |v + omega x r_g|^2 + 1/2 omega.I_g omega."""
    g = np.random.default_rng(6)
    for _ in range(50):
        p = V.params.copy()
        rg = g.uniform(-0.1, 0.1, 3)
        p[I.P_RG:I.P_RG + 3] = rg
        nu = g.normal(size=6)
        v, w = nu[:3], nu[3:]
        vg = v + np.cross(w, rg)
        T_cg = 0.5 * p[I.P_M] * vg @ vg + 0.5 * w @ (p[I.P_IG:I.P_IG + 3] * w)
        np.testing.assert_allclose(0.5 * nu @ O.mass_rb(p) @ nu, T_cg, rtol=1e-13)


# ----------------------------------------------------------------------------- Coriolis

def test_coriolis_skew_symmetric():
    g = np.random.default_rng(7)
    for _ in range(300):
        p = I.perturbed_params(int(g.integers(1 << 30)), V.params, 1)[0]
        p[I.P_RG:I.P_RG + 3] = g.uniform(-0.05, 0.05, 3)
        nu = g.normal(size=6)
        for C in (O.coriolis_rb(p, nu), O.coriolis_a(p, nu)):
            np.testing.assert_allclose(C, -C.T, atol=1e-15)
            assert abs(nu @ C @ nu) <= 1e-13 * (1 + np.abs(C).max() * nu @ nu)


def test_coriolis_rb_matches_newton_euler():
    """About the body origin, the velocity-product terms of the Newton-Euler equations are
    [m(w x v + w x (w x r_g)); w x (I_o w) + m r_g x (w x v)], I_o = I_g - m S(r_g)^2."""
    g = np.random.default_rng(8)
    for _ in range(100):
        p = V.params.copy()
        p[I.P_IG:I.P_IG + 3] = g.uniform(0.1, 0.3, 3)
        rg = g.uniform(-0.1, 0.1, 3)
        p[I.P_RG:I.P_RG + 3] = rg
        m = p[I.P_M]
        nu = g.normal(size=6)
        v, w = nu[:3], nu[3:]
        S = np.array([[0, -rg[2], rg[1]], [rg[2], 0, -rg[0]], [-rg[1], rg[0], 0]])
        Io = np.diag(p[I.P_IG:I.P_IG + 3]) - m * S @ S
        ref = np.concatenate([m * (np.cross(w, v) + np.cross(w, np.cross(w, rg))),
                              np.cross(w, Io @ w) + m * np.cross(rg, np.cross(w, v))])
        np.testing.assert_allclose(O.coriolis_rb(p, nu) @ nu, ref, atol=1e-13)


def test_added_mass_coriolis_munk_moment():
    """Pure translation through the fluid: C_A(nu) nu = [0; v x (M_A,lin v)] (the Munk
    moment), and zero along a principal axis."""
    g = np.random.default_rng(9)
    ma = V.params[I.P_MA:I.P_MA + 3]
    for _ in range(20):
        v = g.normal(size=3)
        nu = np.concatenate([v, np.zeros(3)])
        ref = np.concatenate([np.zeros(3), np.cross(v, ma * v)])
        np.testing.assert_allclose(O.coriolis_a(V.params, nu) @ nu, ref, atol=1e-13)
    nu = np.array([0.7, 0, 0, 0, 0, 0])
    np.testing.assert_allclose(O.coriolis_a(V.params, nu) @ nu, 0, atol=1e-15)


# ----------------------------------------------------------------------------- thrusters

def test_thrust_columns_by_hand():
    s = 1 / math.sqrt(2)
    # thruster 0: at (0.156, -0.111, -0.085) pushing along (s, s, 0), n = 1 -> F = 40 N
    tau = O.thrust(V.params, GEO, [1, 0, 0, 0, 0, 0])
    ref = [40 * s, 40 * s, 0, 0.085 * 40 * s, -0.085 * 40 * s, (0.156 + 0.111) * 40 * s]
    np.testing.assert_allclose(tau, ref, atol=1e-12)
    # thruster 4: vertical at (0, -0.111, 0), n = -0.5 -> F = -10 N along +z (i.e. 10 N up)
    tau = O.thrust(V.params, GEO, [0, 0, 0, 0, -0.5, 0])
    np.testing.assert_allclose(tau, [0, 0, -10, 1.11, 0, 0], atol=1e-12)
    # superposition and the c|c| law
    n = np.array([0.3, -0.2, 0.9, -1.0, 0.4, -0.6])
    cols = np.array([O.thrust(V.params, GEO, np.eye(6)[i]) for i in range(6)]).T
    np.testing.assert_allclose(O.thrust(V.params, GEO, n), cols @ (n * np.abs(n)), atol=1e-12)


def test_allocation_rank():
    def cols(v):
        return np.array([O.thrust(v.params, v.geo(), np.eye(v.n_thr)[i])
                         for i in range(v.n_thr)]).T
    assert np.linalg.matrix_rank(cols(V)) == 5   # pitch tied to surge through the z offset
    assert np.linalg.matrix_rank(cols(VH)) == 6


# ----------------------------------------------------------------------------- RHS

def test_zero_acceleration_at_rest_neutral():
    p = neutral(V.params)
    p[I.P_RG:I.P_RG + 3] = p[I.P_RB:I.P_RB + 3] = (0.01, -0.02, 0.03)
    for q in (np.array([1.0, 0, 0, 0]), quat_from_euler(0.4, -0.3, 1.2)):
        ds = O.rhs(p, GEO, state(p=(3, -1, 2), q=q), np.zeros(6))
        assert np.all(ds == 0.0)


def test_drifting_with_the_current_feels_no_water():
    """A neutral vehicle at rest relative to a constant NED current, not rotating: nu_r = 0, so
    no damping and no added-mass forces; it is carried along at the current's NED velocity."""
    g = np.random.default_rng(10)
    for _ in range(20):
        p = neutral(V.params)
        vc = g.normal(0, 0.3, 3)
        p[I.P_VC:I.P_VC + 3] = vc
        q = quat_from_euler(*g.uniform(-1, 1, 3))
        v = O.rotation(q).T @ vc
        ds = O.rhs(p, GEO, state(q=q, nu=np.concatenate([v, np.zeros(3)])), np.zeros(6))
        np.testing.assert_allclose(ds[I.S_NU:I.S_NU + 6], 0, atol=1e-14)
        np.testing.assert_allclose(ds[I.S_P:I.S_P + 3], vc, atol=1e-14)


def test_quaternion_rate_matches_body_rate():
    """q' = 1/2 q (x) (0, omega): the NED rotation rate R' equals R S(omega)."""
    g = np.random.default_rng(11)
    for _ in range(20):
        q = quat_from_euler(*g.uniform(-1, 1, 3))
        w = g.normal(size=3)
        ds = O.rhs(neutral(V.params), GEO, state(q=q, nu=np.concatenate([np.zeros(3), w])),
                   np.zeros(6))
        qd = ds[I.S_Q:I.S_Q + 4]
        eps = 1e-6
        Rdot = (O.rotation(q + eps * qd) - O.rotation(q - eps * qd)) / (2 * eps)
        Sw = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
        np.testing.assert_allclose(Rdot, O.rotation(q) @ Sw, atol=1e-8)


def test_lag_rk4_exact_discrete_map():
    """n' = (c - n)/tau is linear, so one RK4 step is exactly the 4th-order Taylor polynomial of
    its flow: n1 = c + (n0 - c) P(-h/tau), P(z) = 1 + z + z^2/2 + z^3/6 + z^4/24."""
    p = neutral(V.params)
    n0 = np.array([0.3, -0.7, 0.0, 0.9, -0.1, 0.5])
    c = np.array([-1.0, 1.0, 0.4, 0.9, 0.2, -0.8])
    h = 0.01
    z = -h / p[I.P_TAU]
    P = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    out = O.rk4_step(p, GEO, state(n=n0), c, h)
    np.testing.assert_allclose(out[I.S_N:I.S_N + 6], c + (n0 - c) * P, rtol=1e-14, atol=1e-15)


# ----------------------------------------------------------------------------- closed forms

def test_pure_surge_decay_closed_form():
    p = neutral(V.params)
    a, b, m = p[I.P_DL], p[I.P_DQ], p[I.P_M] + p[I.P_MA]
    u0 = 0.3
    _, traj = rollout1(p, GEO, state(nu=(u0, 0, 0, 0, 0, 0)), [], 500)
    for t in (0.1, 1.0, 5.0):
        e = math.exp(-a * t / m)
        u = a * u0 * e / (a + b * u0 * (1 - e))
        k = int(round(t / 0.01)) - 1
        assert abs(traj[k, I.S_NU] - u) < 1e-9
        assert np.all(traj[k, I.S_NU + 1:I.S_NU + 6] == 0)
    # the printed values of the closed form at t = 0.1, 1, 5 s
    np.testing.assert_allclose(traj[[9, 99, 499], I.S_NU], [0.283969, 0.184099, 0.047274],
                               atol=5e-7)


@pytest.mark.parametrize("F,u_term", [(10.0, 0.639057), (40.0, 1.376613), (80.0, 1.989813)])
def test_terminal_surge_speed(F, u_term):
    p = neutral(V.params)
    p[I.P_KT] = F
    a, b = p[I.P_DL], p[I.P_DQ]
    assert abs((-a + math.sqrt(a * a + 4 * b * F)) / (2 * b) - u_term) < 5e-7
    geo = one_thruster_vehicle()
    s, _ = rollout1(p, geo, state(n=[1.0]), [1.0], 3000)
    assert abs(s[I.S_NU] - u_term) < 2e-6


def test_lag_closed_form():
    p = neutral(V.params)
    _, traj = rollout1(p, GEO, state(n=[0.2] * 6), [0.9, -0.9, 0.5, 0.0, -0.3, 1.0], 40)
    c = np.array([0.9, -0.9, 0.5, 0.0, -0.3, 1.0])
    z = -0.01 / p[I.P_TAU]
    P = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    for k in (4, 19, 39):
        t = (k + 1) * 0.01
        # The thrust moves the vehicle, but n depends only on c and n0: k+1 applications of the
        # exact one-step map, and within RK4's O(h^4) error (h/tau_m = 0.2) of the flow.
        np.testing.assert_allclose(traj[k, I.S_N:I.S_N + 6], c + (0.2 - c) * P ** (k + 1),
                                   rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(traj[k, I.S_N:I.S_N + 6],
                                   c + (0.2 - c) * math.exp(-t / p[I.P_TAU]), atol=2e-5)


def test_pure_yaw_closed_form():
    p = undamped(neutral(V.params))
    r = 0.8
    _, traj = rollout1(p, GEO, state(nu=(0, 0, 0, 0, 0, r)), [], 300)
    for k in (0, 99, 299):
        t = (k + 1) * 0.01
        np.testing.assert_allclose(traj[k, I.S_Q:I.S_Q + 4],
                                   [math.cos(r * t / 2), 0, 0, math.sin(r * t / 2)], atol=1e-12)
        np.testing.assert_allclose(traj[k, I.S_NU + 5], r, atol=1e-14)


def test_constant_velocity_kinematics():
    """Undamped surge with a yawed, pitched attitude: p(t) = R(q0) (u, 0, 0) t."""
    p = undamped(neutral(V.params))
    q0 = quat_from_euler(0.0, 0.3, math.radians(30))
    u = 0.5
    _, traj = rollout1(p, GEO, state(q=q0, nu=(u, 0, 0, 0, 0, 0)), [], 200)
    t = 2.0
    np.testing.assert_allclose(traj[-1, I.S_P:I.S_P + 3], rot_euler(0.0, 0.3, math.radians(30))
                               @ [u * t, 0, 0], atol=1e-12)


# ----------------------------------------------------------------------------- invariants

def _kinetic(p, s):
    nu = s[I.S_NU:I.S_NU + 6]
    return 0.5 * nu @ (O.mass_rb(p) + O.mass_a(p)) @ nu


def _energy(p, s):
    R = O.rotation(s[I.S_Q:I.S_Q + 4])
    G = p[I.P_W] * p[I.P_RG:I.P_RG + 3] - p[I.P_B] * p[I.P_RB:I.P_RB + 3]
    return (_kinetic(p, s) - (p[I.P_W] - p[I.P_B]) * s[I.S_P + 2] - (R @ G)[2])


def _tumbling_state():
    return state(q=quat_from_euler(0.3, -0.2, 0.5), nu=(0.4, -0.3, 0.2, 0.6, -0.5, 0.7))


def _residual_vanishes_4th_order(residual, T=5.0, steps=((0.02, 0.01), (0.01, 0.005)),
                                 small=1e-7):
    """A conserved quantity's drift over [0, T] is pure discretisation error: it must fall at
    least ~14x per halving of h (RK4 is 4th order; a wrong model term gives an O(1) drift that
    does not shrink) and be small at h = 0.01."""
    for h1, h2 in steps:
        e1, e2 = residual(h1, int(round(T / h1))), residual(h2, int(round(T / h2)))
        assert e1 / max(e2, 1e-300) > 14.0, (h1, e1, e2)
        if h1 == 0.01:
            assert e1 < small, e1


def test_energy_conserved_fourth_order():
    """Unforced, undamped, neutral: kinetic energy is conserved by the flow (nu^T C nu = 0)."""
    p = undamped(neutral(V.params))
    p[I.P_IG:I.P_IG + 3] = (0.16, 0.2, 0.25)
    s0 = _tumbling_state()
    T0 = _kinetic(p, s0)

    def drift(h, n):
        _, traj = rollout1(p, GEO, s0, [], n, h=h)
        return max(abs(_kinetic(p, s) - T0) for s in traj[::max(1, n // 20)]) / T0

    _residual_vanishes_4th_order(drift, small=1e-8)


def test_energy_with_restoring_conserved():
    """Undamped, no thrust, no current, W != B and r_g != r_b: T - (W-B) z - e3.R(q)(W r_g -
    B r_b) is conserved."""
    p = undamped(V.params.copy())
    p[I.P_RG:I.P_RG + 3] = (0.01, -0.01, 0.02)
    p[I.P_VC:I.P_VC + 3] = 0.0
    s0 = _tumbling_state()
    E0 = _energy(p, s0)

    def drift(h, n):
        _, traj = rollout1(p, GEO, s0, [], n, h=h)
        return max(abs(_energy(p, s) - E0) for s in traj[::max(1, n // 20)])

    _residual_vanishes_4th_order(drift)
    # the potential actually changed, so the check has teeth
    s, _ = rollout1(p, GEO, s0, [], 500)
    assert abs(_kinetic(p, s) - _kinetic(p, s0)) > 1e-3


def test_impulse_conserved():
    """Kirchhoff: with no external force, the inertial linear impulse R P1 and angular impulse
    R P2 + p x R P1 of [P1; P2] = (M_RB + M_A) nu are constants of motion."""
    p = undamped(neutral(V.params))
    p[I.P_IG:I.P_IG + 3] = (0.16, 0.2, 0.25)
    p[I.P_RG:I.P_RG + 3] = p[I.P_RB:I.P_RB + 3] = (0.01, 0.02, -0.015)
    M = O.mass_rb(p) + O.mass_a(p)

    def impulses(s):
        R = O.rotation(s[I.S_Q:I.S_Q + 4])
        P = M @ s[I.S_NU:I.S_NU + 6]
        L = R @ P[:3]
        return np.concatenate([L, R @ P[3:] + np.cross(s[I.S_P:I.S_P + 3], L)])

    s0 = _tumbling_state()
    J0 = impulses(s0)

    def drift(h, n):
        _, traj = rollout1(p, GEO, s0, [], n, h=h)
        return max(np.abs(impulses(s) - J0).max() for s in traj[::max(1, n // 20)])

    _residual_vanishes_4th_order(drift)


def test_damped_energy_monotone():
    p = neutral(V.params)
    s0 = _tumbling_state()
    _, traj = rollout1(p, GEO, s0, [], 500)
    T = np.array([_kinetic(p, s) for s in traj])
    assert np.all(np.diff(T) <= 1e-14)
    assert T[-1] < 0.05 * T[0]


def test_quaternion_unit_after_each_step():
    p = V.params.copy()
    _, traj = rollout1(p, GEO, _tumbling_state(), [0.5, -0.5, 0.3, 0.9, -0.2, 0.1], 300)
    nq = np.linalg.norm(traj[:, I.S_Q:I.S_Q + 4], axis=1)
    assert np.all(np.abs(nq - 1) < 1e-15)


def test_rk4_order_full_model():
    """Smooth case (no quadratic damping, positive throttle, velocities away from zero): the
    error against a fine Richardson reference falls ~16x per halving of h."""
    p = V.params.copy()
    p[I.P_DQ:I.P_DQ + 6] = 0.0
    p[I.P_VC:I.P_VC + 3] = (0.1, -0.05, 0.02)
    s0 = state(q=quat_from_euler(0.2, 0.1, 0.3), nu=(0.5, 0.2, 0.1, 0.3, 0.2, 0.4),
               n=[0.5] * 6)
    c = [0.6, 0.7, 0.8, 0.5, 0.9, 0.4]
    T = 0.64
    ref, _ = rollout1(p, GEO, s0, c, int(round(T / (0.0025 / 64))), h=0.0025 / 64)
    errs = []
    for h in (0.02, 0.01, 0.005, 0.0025):
        s, _ = rollout1(p, GEO, s0, c, int(round(T / h)), h=h)
        errs.append(np.abs(s - ref).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios > 16 * 0.85) & (ratios < 16 * 1.15)), ratios


def test_current_galilean_invariance():
    """In a current constant in NED, the motion relative to the water is the still-water motion:
    starting from nu_r0, (p - v_c t, q, nu - [R(q)^T v_c; 0]) with the current equals
    (p, q, nu) without it.  Exact for the flow (the added-mass inertia of the current,
    M_A [omega x v_c^b; 0], is what makes it so); RK4's residual vanishes at 4th order."""
    p0 = V.params.copy()
    p0[I.P_VC:I.P_VC + 3] = 0.0
    pc = p0.copy()
    vc = np.array([0.25, -0.15, 0.1])
    pc[I.P_VC:I.P_VC + 3] = vc
    q0 = quat_from_euler(0.3, -0.2, 0.5)
    nu_r0 = np.array([0.4, -0.3, 0.2, 0.6, -0.5, 0.7])
    nu0 = nu_r0 + np.concatenate([O.rotation(q0).T @ vc, np.zeros(3)])
    c = [0.3, -0.4, 0.5, -0.2, 0.6, -0.1]
    T = 2.0

    def residual(h, n, flags=0):
        a, _ = rollout1(p0, GEO, state(q=q0, nu=nu_r0), c, n, h=h, flags=flags)
        b, _ = rollout1(pc, GEO, state(q=q0, nu=nu0), c, n, h=h, flags=flags)
        Rb = O.rotation(b[I.S_Q:I.S_Q + 4])
        rel = b.copy()
        rel[I.S_P:I.S_P + 3] -= vc * (n * h)
        rel[I.S_NU:I.S_NU + 3] -= Rb.T @ vc
        return np.abs(rel - a).max()

    _residual_vanishes_4th_order(residual, T=T, steps=((0.02, 0.01), (0.01, 0.005)), small=1e-8)
    # without the current-acceleration term the relative motion is not the still-water motion
    assert residual(0.01, 200, flags=O.NO_CURRENT_ACCEL) > 1e-4


def test_current_accel_flag_only_matters_when_rotating_in_a_current():
    p = V.params.copy()
    p[I.P_VC:I.P_VC + 3] = (0.2, -0.1, 0.05)
    s = state(q=quat_from_euler(0.1, 0.2, 0.3), nu=(0.1, 0.2, -0.1, 0.3, -0.2, 0.5))
    assert not np.array_equal(O.rhs(p, GEO, s, np.zeros(6)),
                              O.rhs(p, GEO, s, np.zeros(6), flags=O.NO_CURRENT_ACCEL))
    s2 = s.copy()
    s2[I.S_NU + 3:I.S_NU + 6] = 0
    np.testing.assert_array_equal(O.rhs(p, GEO, s2, np.zeros(6)),
                                  O.rhs(p, GEO, s2, np.zeros(6), flags=O.NO_CURRENT_ACCEL))


# ----------------------------------------------------------------------------- randomiser

def test_randomize_distribution_and_determinism():
    from scipy import stats
    n = 20000
    types = np.zeros(n, dtype=np.int32)
    nom = np.stack([V.params, VH.params])
    par = O.randomize(1234, nom, types, 0.8, 1.2, 0.2)
    np.testing.assert_array_equal(par, O.randomize(1234, nom, types, 0.8, 1.2, 0.2))
    ratio = par[:, I.RANDOMISED_INDICES] / V.params[I.RANDOMISED_INDICES]
    assert ratio.min() >= 0.8 and ratio.max() <= 1.2
    assert np.all(np.abs(ratio.mean(0) - 1.0) < 4 * 0.4 / math.sqrt(12 * n))
    for j in range(27):
        assert stats.kstest((ratio[:, j] - 0.8) / 0.4, "uniform").pvalue > 1e-4
    vc = par[:, I.P_VC:I.P_VC + 3]
    for j in range(3):
        assert stats.kstest(vc[:, j] / 0.2, "norm").pvalue > 1e-4
    assert abs(np.corrcoef(vc[:, 0], vc[:, 1])[0, 1]) < 0.05
    # unrandomised entries keep their nominal values
    keep = [i for i in range(I.NPARAM) if i not in I.RANDOMISED_INDICES and
            not I.P_VC <= i < I.P_VC + 3]
    np.testing.assert_array_equal(par[:, keep], np.broadcast_to(V.params[keep], (n, len(keep))))


def test_randomize_keyed_by_global_env_id():
    nom = np.stack([V.params, VH.params])
    types = I.mixed_fleet(7, 300, max_group=40)
    full = O.randomize(99, nom, types)
    part = O.randomize(99, nom, types[100:], gid0=100)
    np.testing.assert_array_equal(full[100:], part)
    # different envs draw differently
    assert np.unique(full[:, I.P_M]).size > 290


def test_reset_draw_distribution():
    from scipy import stats
    z = np.array([O.reset_state(5, 1.0, e, 0)[I.S_NU:I.S_NU + 6] for e in range(4000)])
    for j in range(6):
        assert stats.kstest(z[:, j], "norm").pvalue > 1e-4
    s = O.reset_state(5, 0.3, 17, 3)
    assert s[I.S_Q] == 1.0 and np.all(s[:I.S_Q] == 0) and np.all(s[I.S_N:] == 0)
    assert not np.array_equal(s, O.reset_state(5, 0.3, 17, 4))


def test_procedural_commands_uniform():
    c = np.array([O.commands(11, e, s, 8) for e in range(200) for s in range(10)])
    assert c.min() > -1 and c.max() < 1 and abs(c.mean()) < 0.03
    c6 = O.commands(11, 3, 2, 6)
    assert np.all(c6[6:] == 0) and np.all(c6[:6] == O.commands(11, 3, 2, 8)[:6])


# ----------------------------------------------------------------------------- task layer

def test_euler_angles_invert_quaternion():
    g = np.random.default_rng(21)
    for _ in range(100):
        phi, theta, psi = g.uniform(-3.1, 3.1), g.uniform(-1.5, 1.5), g.uniform(-3.1, 3.1)
        np.testing.assert_allclose(O.euler_zyx(quat_from_euler(phi, theta, psi)),
                                   [phi, theta, psi], atol=1e-12)


def test_task_references_lie_on_their_curves():
    c = np.array([1.0, -2.0, 3.0, 0.7])
    R, w, vz = 2.5, 0.4, 0.15
    for t in np.linspace(0.0, 40.0, 97):
        p = O.task_reference(O.TASK_CIRCLE, c, R, w, vz, t)
        assert abs(np.hypot(p[0] - c[0], p[1] - c[1]) - R) < 1e-12 and p[2] == c[2]
        h = O.task_reference(O.TASK_HELIX, c, R, w, vz, t)
        np.testing.assert_allclose(h[:2], p[:2], atol=1e-15)
        assert abs(h[2] - (c[2] + vz * t)) < 1e-12
        x, y, z = O.task_reference(O.TASK_LEMNISCATE, c, R, w, vz, t) - c[:3]
        assert abs((x * x + y * y) ** 2 - R * R * (x * x - y * y)) < 1e-12 and z == 0
        np.testing.assert_array_equal(O.task_reference(O.TASK_STATION, c, R, w, vz, t), c[:3])
    # periodic with period 2 pi / w
    T = 2 * math.pi / w
    for task in (O.TASK_CIRCLE, O.TASK_LEMNISCATE):
        np.testing.assert_allclose(O.task_reference(task, c, R, w, vz, 3.0),
                                   O.task_reference(task, c, R, w, vz, 3.0 + T), atol=1e-12)


def test_task_observation_and_error():
    c = np.array([1.0, 2.0, -1.0, 0.0])
    s = state(p=(4.0, 6.0, -1.0), q=quat_from_euler(0.1, -0.2, 3.0),
              nu=(0.1, 0.2, 0.3, 0.4, 0.5, 0.6))
    obs, err = O.task_observe(O.TASK_STATION, s, c, 2.0, 0.5, 0.1, -3.0, 4, 0.5, 7.0)
    assert obs.size == 12 and abs(err - 5.0) < 1e-12
    np.testing.assert_allclose(obs[:3], [3.0, 4.0, 0.0])
    # heading error wrapped into (-pi, pi]: 3.0 - (-3.0) = 6.0 -> 6.0 - 2 pi
    np.testing.assert_allclose(obs[3:6], [0.1, -0.2, 6.0 - 2 * math.pi], atol=1e-12)
    np.testing.assert_allclose(obs[6:], [0.1, 0.2, 0.3, 0.4, 0.5, 0.6])
    obs, err = O.task_observe(O.TASK_CIRCLE, s, c, 2.0, 0.5, 0.1, 0.0, 4, 0.5, 7.0)
    assert obs.size == 30
    for i in range(4):
        pr = O.task_reference(O.TASK_CIRCLE, c, 2.0, 0.5, 0.1, 7.0 + (i + 1) * 0.5)
        np.testing.assert_allclose(obs[6 * i:6 * i + 3], s[:3] - pr, atol=1e-12)
    assert abs(err - np.linalg.norm(s[:3] - O.task_reference(O.TASK_CIRCLE, c, 2.0, 0.5, 0.1,
                                                             7.0))) < 1e-12


# ----------------------------------------------------------------------------- split scheme

def split_run(par, geo, s0, c, n_steps, h=0.01, flags=0, xpar=None):
    """Split-scheme sub-steps of one env from rest of the acceleration memory; returns the
    states and accelerations after every sub-step."""
    s, a = s0.copy(), np.zeros(6)
    ss, aa = [], []
    for _ in range(n_steps):
        s, a = O.split_step(par, geo, s, a, c, h, flags, xpar=xpar)
        ss.append(s)
        aa.append(a)
    return np.array(ss), np.array(aa)


def stable_added_mass(par, scale=0.5):
    p = par.copy()
    p[I.P_MA:I.P_MA + 6] *= scale
    return p


def test_split_free_motion_is_semi_implicit_euler():
    """No added mass, damping, restoring force or thrust: the body coasts, p_k = p_0 + k h v
    exactly and q stays put (nothing is lagged when M_A = 0)."""
    par = undamped(neutral(V.params))
    par[I.P_MA:I.P_MA + 6] = 0.0
    v = np.array([0.3, -0.2, 0.1])
    s0 = state(p=(1.0, 2.0, 3.0), nu=(*v, 0, 0, 0))
    ss, aa = split_run(par, GEO, s0, np.zeros(6), 50)
    for k in (1, 10, 50):
        np.testing.assert_allclose(ss[k - 1][I.S_P:I.S_P + 3], [1.0, 2.0, 3.0] + k * 0.01 * v,
                                   rtol=1e-13)
    np.testing.assert_allclose(ss[-1][I.S_Q:I.S_Q + 4], [1, 0, 0, 0], atol=1e-15)
    assert np.abs(aa).max() < 1e-14  # v x (m v) rounds to ~1e-16, not to 0


@pytest.mark.parametrize("ma_scale", [0.5, 1.2])
def test_split_pure_surge_is_the_lagged_linear_recurrence(ma_scale):
    """Pure surge, linear damping d, surge added mass a_m: the lagged added-mass force makes
    a_k = -(d v_k + a_m a_{k-1}) / m and v_{k+1} = v_k + h a_k, i.e. the 2x2 linear map
    [v_{k+1}; a_k] = A [v_k; a_{k-1}], solved here by matrix powers."""
    par = neutral(V.params)
    par[I.P_DQ:I.P_DQ + 6] = 0.0
    m, d = par[I.P_M], par[I.P_DL]
    am = ma_scale * m
    par[I.P_MA] = am
    h, K = 0.01, 120
    ss, aa = split_run(par, GEO, state(nu=(0.4, 0, 0, 0, 0, 0)), np.zeros(6), K, h)
    A = np.array([[1 - h * d / m, -h * am / m], [-d / m, -am / m]])
    x = 0.0
    for k in range(1, K + 1):
        v_k, a_km1 = np.linalg.matrix_power(A, k) @ np.array([0.4, 0.0])
        x += h * v_k  # semi-implicit: the position moves with the new velocity
        if k in (1, 7, 60, K):
            np.testing.assert_allclose(ss[k - 1][I.S_NU], v_k, rtol=1e-10, atol=1e-13)
            np.testing.assert_allclose(aa[k - 1][0], a_km1, rtol=1e-10, atol=1e-13)
            np.testing.assert_allclose(ss[k - 1][I.S_P], x, rtol=1e-10, atol=1e-13)
    # the lagged added-mass mode has eigenvalue ~ -a_m/m: it dies out for a_m < m and grows
    # (alternating in sign) for a_m > m, at the rate of A's dominant eigenvalue
    lam = np.linalg.eigvals(A)
    mode = lam[np.argmin(lam.real)]
    assert abs(mode + am / m) < 0.02
    if ma_scale > 1:
        r = aa[K - 1][0] / aa[K - 2][0]
        assert abs(r - mode.real) < 1e-6 and abs(aa[K - 1][0]) > 1e3 * abs(aa[0][0])


def test_split_pure_yaw_attitude_update():
    """Pure yaw with linear yaw damping and no added mass: r_k = r_0 (1 - h d / I)^k, and the
    normalised update q + h/2 q (x) (0, 0, 0, r_k) turns the heading by 2 atan(h r_k / 2) with
    the new rate r_k."""
    par = neutral(V.params)
    par[I.P_MA:I.P_MA + 6] = 0.0
    par[I.P_DQ:I.P_DQ + 6] = 0.0
    d, Iz, h, r0 = par[I.P_DL + 5], par[I.P_IG + 2], 0.01, 0.8
    ss, _ = split_run(par, GEO, state(nu=(0, 0, 0, 0, 0, r0)), np.zeros(6), 200, h)
    psi = 0.0
    for k in range(1, 201):
        r_k = r0 * (1 - h * d / Iz) ** k
        psi += 2 * math.atan(h * r_k / 2)
        if k in (1, 50, 200):
            np.testing.assert_allclose(ss[k - 1][I.S_NU + 5], r_k, rtol=1e-12)
            q = ss[k - 1][I.S_Q:I.S_Q + 4]
            np.testing.assert_allclose(q, [math.cos(psi / 2), 0, 0, math.sin(psi / 2)],
                                       atol=1e-12)


def test_split_equilibrium_equals_the_coupled_one():
    """At a steady state nu' = 0 and the lagged acceleration is 0, so the split scheme's fixed
    point is the coupled Eq. 1's equilibrium: held throttles, both integrated to rest."""
    par = stable_added_mass(V.params, 0.5)
    c = np.array([0.6, 0.6, -0.6, -0.6, 0.3, -0.3])
    ss, aa = split_run(par, GEO, state(), c, 10000)
    s_rk4, _ = rollout1(par, GEO, state(), c, 10000)
    assert np.abs(aa[-1]).max() < 1e-9
    # (the held throttles spin the vehicle about the vertical: nu is steady, the heading is not,
    # so the two runs' headings differ by their phase error and nu agrees to ~3e-8)
    np.testing.assert_allclose(ss[-1][I.S_NU:I.S_NU + 6], s_rk4[I.S_NU:I.S_NU + 6], rtol=1e-6,
                               atol=1e-8)


def test_split_converges_to_the_coupled_solution_at_first_order():
    """With every added mass below the rigid-body mass the split scheme is stable and its error
    against the coupled equation (RK4 at a fine step) halves with h: first order."""
    par = stable_added_mass(V.params, 0.5)
    par[I.P_VC:I.P_VC + 3] = [0.1, -0.05, 0.02]
    c = np.array([0.5, -0.3, 0.2, 0.4, -0.6, 0.1])
    s0 = state(q=quat_from_euler(0.2, -0.1, 0.5), nu=(0.2, -0.1, 0.05, 0.1, -0.2, 0.15))
    T = 1.0
    ref, _ = rollout1(par, GEO, s0, c, 4000, h=T / 4000)
    errs = []
    for h in (0.01, 0.005, 0.0025):
        ss, _ = split_run(par, GEO, s0, c, int(round(T / h)), h)
        errs.append(np.abs(ss[-1][I.S_NU:I.S_NU + 6] - ref[I.S_NU:I.S_NU + 6]).max())
    for e1, e2 in zip(errs, errs[1:]):
        assert 1.7 < e1 / e2 < 2.3, errs


def split_general_case(kind):
    """Off-centre gravity and / or a full M_A and D_l, with every added mass small enough for the
    lagged added-mass mode to decay (spectral radius of M_RB^-1 M_A below 0.6)."""
    par = stable_added_mass(V.params, 0.35)
    par[I.P_VC:I.P_VC + 3] = [0.1, -0.05, 0.02]
    xpar = None
    g = np.random.default_rng(17)
    if kind in ("rg", "both"):
        par[I.P_RG:I.P_RG + 3] = [0.012, -0.018, 0.02]
    if kind in ("full", "both"):
        ma, dl = par[I.P_MA:I.P_MA + 6], par[I.P_DL:I.P_DL + 6]
        U = g.uniform(-1, 1, (6, 6))
        MA = np.diag(ma) + 0.12 * (U + U.T) / 2 * np.sqrt(np.outer(ma, ma)) * (1 - np.eye(6))
        DL = np.diag(dl) + 0.12 * g.uniform(-1, 1, (6, 6)) * np.sqrt(np.outer(dl, dl)) * (
            1 - np.eye(6))
        xpar = xpar_from_matrices(MA, DL)
    rho = np.abs(np.linalg.eigvals(np.linalg.solve(O.mass_rb(par), O.mass_a(par, xpar)))).max()
    assert rho < 0.6, rho
    return par, xpar


@pytest.mark.parametrize("kind", ["rg", "full", "both"])
def test_split_general_model_converges_to_the_coupled_solution_at_first_order(kind):
    """The split scheme with the full rigid-body inertia (r_g off the origin: M_RB couples
    surge, sway and heave to the rotations, C_RB carries the m r_g terms and the weight a
    moment) and the full M_A and D_l converges to the coupled equation with the same terms at
    first order: any term dropped or mis-signed on one side changes the limit."""
    par, xpar = split_general_case(kind)
    c = np.array([0.5, -0.3, 0.2, 0.4, -0.6, 0.1])
    s0 = state(q=quat_from_euler(0.2, -0.1, 0.5), nu=(0.2, -0.1, 0.05, 0.1, -0.2, 0.15))
    T = 1.0
    ref, _ = rollout1(par, GEO, s0, c, 4000, h=T / 4000, xpar=xpar)
    errs = []
    for h in (0.01, 0.005, 0.0025):
        ss, _ = split_run(par, GEO, s0, c, int(round(T / h)), h, xpar=xpar)
        errs.append(np.abs(ss[-1][I.S_NU:I.S_NU + 6] - ref[I.S_NU:I.S_NU + 6]).max())
    for e1, e2 in zip(errs, errs[1:]):
        assert 1.7 < e1 / e2 < 2.3, errs
    assert errs[-1] < 5e-3, errs


def test_split_general_model_equilibrium_equals_the_coupled_one():
    """Held throttles, off-centre gravity, full M_A and D_l: at rest of the acceleration memory
    the split scheme's fixed point is the coupled equation's steady state."""
    par, xpar = split_general_case("both")
    par[I.P_VC:I.P_VC + 3] = 0.0
    c = np.array([0.6, 0.6, -0.6, -0.6, 0.3, -0.3])
    ss, aa = split_run(par, GEO, state(), c, 10000, xpar=xpar)
    s_rk4, _ = rollout1(par, GEO, state(), c, 10000, xpar=xpar)
    assert np.abs(aa[-1]).max() < 1e-8
    np.testing.assert_allclose(ss[-1][I.S_NU:I.S_NU + 6], s_rk4[I.S_NU:I.S_NU + 6], rtol=1e-6,
                               atol=1e-8)


def test_split_step_defaults_to_the_diagonal_extension():
    """xpar = None and an all-zero extension give the same split sub-step, bit for bit."""
    par, _ = split_general_case("rg")
    s0 = state(q=quat_from_euler(0.3, 0.1, -0.4), nu=(0.2, 0.1, -0.1, 0.2, 0.1, -0.3),
               n=(0.2, -0.4, 0.1, 0.3, -0.2, 0.5))
    a0 = np.array([0.1, -0.2, 0.05, 0.3, -0.1, 0.2])
    c = np.array([0.5, -0.3, 0.2, 0.4, -0.6, 0.1])
    s1, a1 = O.split_step(par, GEO, s0, a0, c, 0.01)
    s2, a2 = O.split_step(par, GEO, s0, a0, c, 0.01, xpar=np.zeros(O.NXPARAM))
    assert np.array_equal(s1, s2) and np.array_equal(a1, a2)


# ----------------------------------------------------------------------------- full M_A and D

def xpar_from_matrices(MA, DL):
    """Pack a full symmetric M_A and a full D_l into the off-diagonal extension: M_A above the
    diagonal row-major, then D_l's off-diagonal entries row-major."""
    up = [MA[i, j] for i in range(6) for j in range(i + 1, 6)]
    off = [DL[i, j] for i in range(6) for j in range(6) if j != i]
    return np.array(up + off)


def random_hydro(g, par):
    """A random symmetric positive-definite M_A and a D_l with positive-definite symmetric part,
    keeping the record's diagonals (so that the two stay consistent)."""
    A = g.normal(size=(6, 6)) * 0.3
    MA = A @ A.T + np.diag(par[I.P_MA:I.P_MA + 6])
    B = g.normal(size=(6, 6)) * 0.4
    DL = B @ B.T + np.diag(par[I.P_DL:I.P_DL + 6]) + 0.5 * (g.normal(size=(6, 6)) -
                                                             g.normal(size=(6, 6)).T)
    p = par.copy()
    p[I.P_MA:I.P_MA + 6] = np.diag(MA)
    p[I.P_DL:I.P_DL + 6] = np.diag(DL)
    return p, MA, DL


def test_extension_layout_builds_the_full_matrices():
    g = np.random.default_rng(3)
    p, MA, DL = random_hydro(g, V.params)
    x = xpar_from_matrices(MA, DL)
    np.testing.assert_array_equal(O.mass_a(p, x), MA)
    nu = g.normal(size=6)
    want = DL + np.diag(p[I.P_DQ:I.P_DQ + 6] * np.abs(nu))
    np.testing.assert_allclose(O.damping(p, nu, x), want, rtol=1e-15, atol=1e-15)
    # a zero extension is the diagonal model
    np.testing.assert_array_equal(O.mass_a(V.params, np.zeros(O.NXPARAM)), O.mass_a(V.params))


def test_full_added_mass_coriolis_skew_symmetric():
    g = np.random.default_rng(11)
    for _ in range(200):
        p, MA, DL = random_hydro(g, V.params)
        x = xpar_from_matrices(MA, DL)
        nu = g.normal(size=6)
        C = O.coriolis_a(p, nu, x)
        np.testing.assert_allclose(C, -C.T, atol=1e-15)
        assert abs(nu @ C @ nu) <= 1e-13 * (1 + np.abs(C).max() * nu @ nu)


def test_full_hydro_power_balance():
    """No current, thrust or restoring force: d/dt (1/2 nu^T M nu) = nu^T M nu' must equal
    -nu^T D(nu) nu (the Coriolis terms do no work), with M = M_RB + M_A and D built here from
    the extension's documented layout, r_g off centre."""
    g = np.random.default_rng(12)
    for _ in range(100):
        p, MA, DL = random_hydro(g, neutral(V.params))
        p[I.P_RG:I.P_RG + 3] = g.uniform(-0.03, 0.03, 3)
        p[I.P_RB:I.P_RB + 3] = p[I.P_RG:I.P_RG + 3]
        x = xpar_from_matrices(MA, DL)
        nu = g.normal(size=6)
        ds = O.rhs(p, GEO, state(q=quat_from_euler(*g.uniform(-1, 1, 3)), nu=nu), np.zeros(6),
                   xpar=x)
        M = O.mass_rb(p) + MA
        D = DL + np.diag(p[I.P_DQ:I.P_DQ + 6] * np.abs(nu))
        lhs = nu @ M @ ds[I.S_NU:I.S_NU + 6]
        assert abs(lhs + nu @ D @ nu) <= 1e-12 * (1 + abs(nu @ D @ nu))


def test_full_added_mass_energy_conserved_undamped():
    """Undamped, neutral, no thrust: Kirchhoff's equations with a full M_A conserve
    T = 1/2 nu^T (M_RB + M_A) nu; RK4's drift over 1 s is tiny and falls ~16x per halving."""
    g = np.random.default_rng(13)
    p, MA, _ = random_hydro(g, neutral(V.params))
    p = undamped(p)
    x = xpar_from_matrices(MA, np.zeros((6, 6)))
    M = O.mass_rb(p) + MA
    s0 = state(nu=(0.4, -0.3, 0.2, 0.8, -0.6, 0.5))
    T0 = 0.5 * s0[I.S_NU:I.S_NU + 6] @ M @ s0[I.S_NU:I.S_NU + 6]
    drift = []
    for h in (0.02, 0.01):
        s, _ = O.rollout(p[None], GEO[None], [0], s0[None], np.zeros((1, 1, 8)), 1,
                         int(round(1.0 / h)), h=h, record=True, xpar=x[None])
        nu = s[0, I.S_NU:I.S_NU + 6]
        drift.append(abs(0.5 * nu @ M @ nu - T0) / T0)
    assert drift[1] < 1e-8 and drift[0] / drift[1] > 10, drift


def test_randomize_centre_of_gravity():
    from scipy import stats
    n = 20000
    types = np.zeros(n, dtype=np.int32)
    nom = np.stack([V.params, VH.params])
    par = O.randomize(1234, nom, types, 0.8, 1.2, 0.2, rg_halfwidth=0.02)
    base = O.randomize(1234, nom, types, 0.8, 1.2, 0.2)
    # only r_g changes, and it is nominal + U[-w, w] per axis, independent across axes
    others = [i for i in range(I.NPARAM) if not I.P_RG <= i < I.P_RG + 3]
    np.testing.assert_array_equal(par[:, others], base[:, others])
    d = par[:, I.P_RG:I.P_RG + 3] - V.params[I.P_RG:I.P_RG + 3]
    assert np.abs(d).max() <= 0.02
    for j in range(3):
        assert stats.kstest((d[:, j] + 0.02) / 0.04, "uniform").pvalue > 1e-4
    assert abs(np.corrcoef(d[:, 0], d[:, 2])[0, 1]) < 0.05


def test_full_added_mass_impulse_conserved():
    """Kirchhoff: for the unforced body in still water the impulses of P = (M_RB + M_A) nu are
    constant in the inertial frame, linear R(q) P1 and angular R(q) P2 + p x R(q) P1, only if
    the Coriolis terms are built from the same full M_A as the inertia (energy alone cannot
    tell)."""
    g = np.random.default_rng(14)
    p, MA, _ = random_hydro(g, neutral(V.params))
    p = undamped(p)
    p[I.P_RG:I.P_RG + 3] = [0.01, -0.02, 0.015]
    p[I.P_RB:I.P_RB + 3] = p[I.P_RG:I.P_RG + 3]
    x = xpar_from_matrices(MA, np.zeros((6, 6)))
    M = O.mass_rb(p) + MA
    s0 = state(q=quat_from_euler(0.3, -0.2, 0.7), nu=(0.4, -0.3, 0.2, 0.8, -0.6, 0.5))

    def impulses(s):
        R = O.rotation(s[I.S_Q:I.S_Q + 4])
        P = M @ s[I.S_NU:I.S_NU + 6]
        L = R @ P[:3]
        return np.r_[L, R @ P[3:] + np.cross(s[I.S_P:I.S_P + 3], L)]

    s, _ = O.rollout(p[None], GEO[None], [0], s0[None], np.zeros((1, 1, 8)), 1, 200, h=0.005,
                     record=True, xpar=x[None])
    np.testing.assert_allclose(impulses(s[0]), impulses(s0), rtol=0, atol=1e-8)
