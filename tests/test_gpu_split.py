"""Split-integration comparison step (§METHOD's engine + hydrodynamics-module arrangement) on the
GPU against the FP64 oracle's split scheme: one teacher-forced sub-step with a non-zero
acceleration memory, stable rollouts, the unstable added-mass mode, and launch-shape
invariance, for diagonal-mass fleets and on the general model (off-centre gravity, full M_A and
D_l)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2410_14117_gb300 import inputs as I
from paper_2410_14117_gb300.sim import MGError, Sim

from _helpers import TOL_ROLLOUT, TOL_STEP, oracle_geo, oracle_nominal, rel_err, vehicles

pytestmark = pytest.mark.gpu

H = 0.01


def _params(seed, types, vs, ma_scale):
    p = I.perturbed_params(seed, oracle_nominal(vs)[types], len(types))
    p[:, I.P_MA:I.P_MA + 6] = I.round_f32(p[:, I.P_MA:I.P_MA + 6] * ma_scale)
    return p


def _general(seed, params, kind, coupling=0.15):
    """Off-centre gravity (r_g ~ U[-2, 2] cm) and / or the off-diagonal extension."""
    p = params.copy()
    xpar = None
    if kind in ("rg", "both"):
        p[:, I.P_RG:I.P_RG + 3] = I.round_f32(
            np.random.default_rng(seed).uniform(-0.02, 0.02, (len(p), 3)))
    if kind in ("full", "both"):
        xpar = I.hydro_offdiag(seed + 1, p, coupling)
    return p, xpar


def _sim(types, vs, params, states, accel, epb=128, spl=50, xpar=None):
    sim = Sim(len(types), types, vs)
    sim.set_launch(epb, spl, False)
    sim.set_params(torch.tensor(params, dtype=torch.float32, device="cuda"))
    if xpar is not None:
        sim.set_hydro_offdiag(torch.tensor(xpar, dtype=torch.float32, device="cuda"))
    sim.set_state(torch.tensor(states, dtype=torch.float32, device="cuda"))
    acc = torch.tensor(np.ascontiguousarray(accel.T), dtype=torch.float32, device="cuda")
    return sim, acc


def _acc_err(got, ref):
    """Per env: |a_gpu - a_ref|_inf / max(|a_ref|_inf, 0.1)."""
    return np.abs(got - ref).max(axis=1) / np.maximum(np.abs(ref).max(axis=1), 0.1)


@pytest.mark.parametrize("flags", [0, 1])
def test_split_one_substep_matches_oracle(flags):
    vs = vehicles()
    n = 3000
    types = I.mixed_fleet(31, n, max_group=400)
    nt = np.array([vs[t].n_thr for t in types])
    params = _params(32, types, vs, 1.0)
    states = I.random_states(33, n, nt)
    accel = I.round_f32(np.random.default_rng(34).normal(0.0, 0.5, (n, 6)))
    cmds = I.commands(35, 1, n, nt)
    sim, acc = _sim(types, vs, params, states, accel)
    sim.set_model_flags(flags)
    sim.set_actions(torch.tensor(cmds, device="cuda"), 1)
    sim.step_split(1, acc)
    got = sim.get_state().double().cpu().numpy()
    got_a = acc.double().cpu().numpy().T
    sim.close()
    geo = oracle_geo(vs)
    for e in range(n):
        s_ref, a_ref = O.split_step(params[e], geo[types[e]], states[e], accel[e],
                                    cmds[0, e], H, flags)
        assert rel_err(got[e][None], s_ref[None]).max() <= TOL_STEP, e
        assert _acc_err(got_a[e][None], a_ref[None]).max() <= TOL_STEP, e


@pytest.mark.parametrize("flags", [0, 1])
@pytest.mark.parametrize("kind", ["rg", "full", "both"])
def test_split_general_one_substep_matches_oracle(kind, flags):
    vs = vehicles()
    n = 3000
    types = I.mixed_fleet(131, n, max_group=400)
    nt = np.array([vs[t].n_thr for t in types])
    params, xpar = _general(136, _params(132, types, vs, 1.0), kind)
    states = I.random_states(133, n, nt)
    accel = I.round_f32(np.random.default_rng(134).normal(0.0, 0.5, (n, 6)))
    cmds = I.commands(135, 1, n, nt)
    sim, acc = _sim(types, vs, params, states, accel, xpar=xpar)
    sim.set_model_flags(flags)
    sim.set_actions(torch.tensor(cmds, device="cuda"), 1)
    sim.step_split(1, acc)
    got = sim.get_state().double().cpu().numpy()
    got_a = acc.double().cpu().numpy().T
    sim.close()
    geo = oracle_geo(vs)
    for e in range(n):
        s_ref, a_ref = O.split_step(params[e], geo[types[e]], states[e], accel[e], cmds[0, e],
                                    H, flags, xpar=None if xpar is None else xpar[e])
        assert rel_err(got[e][None], s_ref[None]).max() <= TOL_STEP, e
        assert _acc_err(got_a[e][None], a_ref[None]).max() <= TOL_STEP, e


def test_split_general_stable_rollout_matches_oracle():
    """Off-centre gravity with a 10 %-coupled M_A and D_l, added mass scaled by 0.4 (every env's
    lagged added-mass mode decays: spectral radius of M_RB^-1 M_A below 1): 300 sub-steps."""
    vs = vehicles()
    n = 1024
    types = I.mixed_fleet(141, n, max_group=300)
    nt = np.array([vs[t].n_thr for t in types])
    params, xpar = _general(146, _params(142, types, vs, 0.4), "both", coupling=0.1)
    rho = max(np.abs(np.linalg.eigvals(np.linalg.solve(O.mass_rb(params[e]),
                                                       O.mass_a(params[e], xpar[e])))).max()
              for e in range(n))
    assert rho < 0.95, rho
    states = I.initial_states(143, n)
    for e in range(n):
        states[e, I.S_N + nt[e]:] = 0.0
    cmds = I.commands(144, 30, n, nt)
    sim, acc = _sim(types, vs, params, states, np.zeros((n, 6)), spl=64, xpar=xpar)
    sim.set_actions(torch.tensor(cmds, device="cuda"), 10)
    sim.step_split(300, acc)
    assert sim.sync() == 0
    got = sim.get_state().double().cpu().numpy()
    got_a = acc.double().cpu().numpy().T
    sim.close()
    ref, ref_a = O.split_rollout(params, oracle_geo(vs), types, states, np.zeros((n, 6)),
                                 cmds.astype(np.float64), 10, 300, h=H, xpar=xpar)
    err = rel_err(got, ref)
    assert err.max() <= TOL_ROLLOUT, err.max(axis=0)
    assert _acc_err(got_a, ref_a).max() <= 10 * TOL_ROLLOUT


def test_split_stable_rollout_matches_oracle():
    """Added mass halved (every ratio to the rigid-body mass below 1: the scheme is stable):
    300 sub-steps with held commands and currents."""
    vs = vehicles()
    n = 1024
    types = I.mixed_fleet(41, n, max_group=300)
    nt = np.array([vs[t].n_thr for t in types])
    params = _params(42, types, vs, 0.5)
    states = I.initial_states(43, n)
    for e in range(n):
        states[e, I.S_N + nt[e]:] = 0.0
    cmds = I.commands(44, 30, n, nt)
    sim, acc = _sim(types, vs, params, states, np.zeros((n, 6)), spl=64)
    sim.set_actions(torch.tensor(cmds, device="cuda"), 10)
    sim.step_split(300, acc)
    assert sim.sync() == 0
    got = sim.get_state().double().cpu().numpy()
    got_a = acc.double().cpu().numpy().T
    sim.close()
    ref, ref_a = O.split_rollout(params, oracle_geo(vs), types, states, np.zeros((n, 6)),
                                 cmds.astype(np.float64), 10, 300, h=H)
    err = rel_err(got, ref)
    assert err.max() <= TOL_ROLLOUT, err.max(axis=0)
    assert _acc_err(got_a, ref_a).max() <= 10 * TOL_ROLLOUT


def test_split_unstable_added_mass_mode_grows_as_predicted():
    """Nominal BlueROV2: heave added mass 14.57 kg over a rigid-body mass of 11.5 kg, so the
    lagged added-mass force feeds a heave-acceleration mode with factor ~ -14.57/11.5 per
    sub-step.  The GPU follows the oracle while the mode is young (20 sub-steps from random
    velocities), and in pure heave the mode's growth per sub-step matches the prediction."""
    vs = vehicles()
    n = 256
    types = np.zeros(n, dtype=np.int32)
    params = np.repeat(oracle_nominal(vs)[:1], n, axis=0)
    states = I.initial_states(51, n)
    sim, acc = _sim(types, vs, params, states, np.zeros((n, 6)))
    sim.set_actions(None, 1)
    sim.step_split(20, acc)
    got = sim.get_state().double().cpu().numpy()
    got_a = acc.double().cpu().numpy().T
    sim.close()
    ref, ref_a = O.split_rollout(params, oracle_geo(vs), types, states, np.zeros((n, 6)),
                                 np.zeros((1, n, 8)), 1, 20, h=H)
    assert rel_err(got, ref).max() <= TOL_ROLLOUT
    assert _acc_err(got_a, ref_a).max() <= 10 * TOL_ROLLOUT
    # pure heave from w0 in [-0.5, 0.5] with linear damping only: the attitude stays level and
    # a_k follows the linear recurrence of the oracle pin, whose dominant eigenvalue is
    # ~ -m_a / m; after 30 sub-steps the acceleration's ratio per sub-step is that eigenvalue
    lin = params.copy()
    lin[:, I.P_DQ:I.P_DQ + 6] = 0.0
    heave = np.zeros((n, I.NSTATE))
    heave[:, I.S_Q] = 1.0
    heave[:, I.S_NU + 2] = I.round_f32(np.linspace(-0.5, 0.5, n))
    sim, acc = _sim(types, vs, lin, heave, np.zeros((n, 6)))
    sim.set_actions(None, 1)
    sim.step_split(30, acc)
    a30 = acc.double().cpu().numpy().T.copy()
    sim.step_split(1, acc)
    a31 = acc.double().cpu().numpy().T
    sim.close()
    m, ma, d = lin[0, I.P_M], lin[0, I.P_MA + 2], lin[0, I.P_DL + 2]
    lam = np.linalg.eigvals(np.array([[1 - H * d / m, -H * ma / m], [-d / m, -ma / m]]))
    dominant = lam[np.argmax(np.abs(lam))].real
    assert dominant < -1.2
    np.testing.assert_allclose(a31[:, 2] / a30[:, 2], dominant, rtol=5e-3)
    assert np.abs(a30[:, [0, 1, 3, 4, 5]]).max() == 0.0


@pytest.mark.parametrize("kind", ["diag", "both"])
def test_split_launch_shape_and_errors(kind):
    """Chunked launches (sub-steps per launch, block size) give the same bits, for a diagonal-
    mass fleet and on the general model; a host accel buffer is rejected on the host."""
    vs = vehicles()
    n = 1000
    types = I.mixed_fleet(61, n, max_group=200)
    nt = np.array([vs[t].n_thr for t in types])
    params, xpar = _general(67, _params(62, types, vs, 0.5), kind, coupling=0.1)
    states = I.initial_states(63, n)
    for e in range(n):
        states[e, I.S_N + nt[e]:] = 0.0
    cmds = torch.tensor(I.commands(64, 12, n, nt), device="cuda")
    out = []
    for epb, spl, calls in ((128, 50, (120,)), (64, 7, (33, 80, 7)), (256, 1, (120,))):
        sim, acc = _sim(types, vs, params, states, np.zeros((n, 6)), epb=epb, spl=spl,
                        xpar=xpar)
        sim.set_actions(cmds, 10)
        for k in calls:
            sim.step_split(k, acc)
        out.append((sim.get_state().cpu(), acc.cpu()))
        sim.close()
    for s, a in out[1:]:
        assert torch.equal(s, out[0][0]) and torch.equal(a, out[0][1])
    sim, _ = _sim(np.zeros(8, np.int32), vs, _params(65, np.zeros(8, np.int32), vs, 0.5),
                  I.initial_states(66, 8), np.zeros((8, 6)))
    with pytest.raises((MGError, ValueError)):
        sim.step_split(1, torch.zeros((6, 8)))
    sim.close()
