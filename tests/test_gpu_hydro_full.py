"""Full (non-diagonal) added mass and linear damping, and randomised centres of gravity, on the
GPU against the FP64 oracle: one teacher-forced sub-step, 500-sub-step rollouts, the extension's
round trip, the randomiser's r_g draw, and the paths that must accept or reject the extension."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2410_14117_gb300 import inputs as I
from paper_2410_14117_gb300._lib import call
from paper_2410_14117_gb300.sim import MGError, Sim

from _helpers import (TOL_QNORM, TOL_ROLLOUT, TOL_STEP, f32, oracle_geo, oracle_nominal,
                      rel_err, vehicles)

pytestmark = pytest.mark.gpu

H = 0.01


def _fleet(seed, n, vs, rg=0.02):
    types = I.mixed_fleet(seed, n, max_group=300)
    params = I.perturbed_params(seed + 1, oracle_nominal(vs)[types], n)
    g = np.random.default_rng(seed + 2)
    params[:, I.P_RG:I.P_RG + 3] = I.round_f32(g.uniform(-rg, rg, (n, 3)))
    xpar = I.hydro_offdiag(seed + 3, params)
    return types, params, xpar


def _sim(types, vs, params, xpar, states, epb=128, spl=50, queue=False):
    sim = Sim(len(types), types, vs)
    sim.set_launch(epb, spl, True)
    sim.set_schedule(queue)
    sim.set_params(torch.tensor(params, dtype=torch.float32, device="cuda"))
    sim.set_hydro_offdiag(torch.tensor(xpar, dtype=torch.float32, device="cuda"))
    sim.set_state(torch.tensor(states, dtype=torch.float32, device="cuda"))
    return sim


@pytest.mark.parametrize("flags", [0, 1])
def test_full_hydro_one_substep_matches_oracle(flags):
    vs = vehicles()
    n = 4096
    types, params, xpar = _fleet(71, n, vs)
    nt = np.array([vs[t].n_thr for t in types])
    states = I.random_states(75, n, nt)
    cmds = I.commands(76, 1, n, nt)
    sim = _sim(types, vs, params, xpar, states)
    sim.set_model_flags(flags)
    sim.set_actions(torch.tensor(cmds, device="cuda"), 1)
    sim.step(1)
    got = sim.get_state().double().cpu().numpy()
    sim.close()
    ref = O.rollout(params, oracle_geo(vs), types, states, cmds.astype(np.float64), 1, 1, h=H,
                    flags=flags, xpar=xpar)
    err = rel_err(got, ref)
    assert err.max() <= TOL_STEP, err.max(axis=0)


@pytest.mark.parametrize("epb,spl", [(128, 50), (64, 1), (256, 500)])
def test_full_hydro_500_substeps_matches_oracle(epb, spl):
    vs = vehicles()
    n = 1024
    types, params, xpar = _fleet(81, n, vs)
    nt = np.array([vs[t].n_thr for t in types])
    states = I.initial_states(85, n)
    for e in range(n):
        states[e, I.S_N + nt[e]:] = 0.0
    cmds = I.commands(86, 50, n, nt)
    sim = _sim(types, vs, params, xpar, states, epb=epb, spl=spl)
    sim.set_actions(torch.tensor(cmds, device="cuda"), 10)
    traj = sim.step_record(500).cpu().numpy().astype(np.float64)
    got = sim.get_state().double().cpu().numpy()
    assert sim.sync() == 0
    sim.close()
    ref = O.rollout(params, oracle_geo(vs), types, states, cmds.astype(np.float64), 10, 500,
                    h=H, xpar=xpar)
    err = rel_err(got, ref)
    assert err.max() <= TOL_ROLLOUT, err.max(axis=0)
    assert np.abs(np.linalg.norm(traj[:, 3:7, :], axis=1) - 1.0).max() <= TOL_QNORM


def test_extension_round_trip_clear_and_schedules():
    """get returns what was set; clearing gives the diagonal model bit for bit; the work-queue
    schedule (its off-diagonal variant), graph replay and mg_step_noalloc give the static grid's
    bits; the task step carries the extension."""
    vs = vehicles()
    n = 1500
    types, params, xpar = _fleet(91, n, vs, rg=0.0)
    states = I.initial_states(95, n)
    nt = np.array([vs[t].n_thr for t in types])
    for e in range(n):
        states[e, I.S_N + nt[e]:] = 0.0
    sim = _sim(types, vs, params, xpar, states)
    np.testing.assert_array_equal(sim.get_hydro_offdiag().cpu().numpy(),
                                  xpar.astype(np.float32))
    sim.set_procedural_actions(7, 10)
    sim.step(120)
    a = sim.get_state().cpu()
    sim.close()
    sim = _sim(types, vs, params, xpar, states, epb=64, spl=7, queue=True)
    sim.set_procedural_actions(7, 10)
    for _ in range(12):
        sim.step(10)
    torch.testing.assert_close(sim.get_state().cpu(), a, rtol=0, atol=0)
    # the no-allocation entry point runs the same work-queue kernel
    sim.set_state(torch.tensor(states, dtype=torch.float32, device="cuda"))
    sim.set_procedural_actions(7, 10)
    for _ in range(12):
        call("mg_step_noalloc", sim._h, 10)
    torch.testing.assert_close(sim.get_state().cpu(), a, rtol=0, atol=0)
    # cleared: the same as a sim that never had the extension
    sim.set_hydro_offdiag(None)
    assert not sim.get_hydro_offdiag().any()
    sim.set_state(torch.tensor(states, dtype=torch.float32, device="cuda"))
    sim.set_procedural_actions(7, 10)
    sim.step(120)
    b = sim.get_state().cpu()
    sim.close()
    plain = Sim(n, types, vs)
    plain.set_params(torch.tensor(params, dtype=torch.float32, device="cuda"))
    plain.set_state(torch.tensor(states, dtype=torch.float32, device="cuda"))
    plain.set_procedural_actions(7, 10)
    plain.step(120)
    torch.testing.assert_close(plain.get_state().cpu(), b, rtol=0, atol=0)
    plain.close()
    assert not torch.equal(a, b)
    # the fused task step runs the same sub-steps
    outs = []
    for task in (False, True):
        sim = _sim(types, vs, params, xpar, states)
        sim.set_procedural_actions(7, 10)
        if task:
            sim.set_task(0, torch.zeros((n, 4), device="cuda"), max_error=0.0, episode_steps=0)
            sim.task_step(10)
        else:
            sim.step(10)
        outs.append(sim.get_state().cpu())
        sim.close()
    torch.testing.assert_close(outs[1], outs[0], rtol=0, atol=0)


def test_randomized_centre_of_gravity_matches_oracle():
    vs = vehicles()
    n = 2048
    types = I.mixed_fleet(101, n, max_group=500)
    sim = Sim(n, types, vs)
    sim.randomize(4242, 0.8, 1.2, 0.2, 0.3, rg_halfwidth=0.02)
    got = sim.get_params().double().cpu().numpy()
    ref = I.round_f32(O.randomize(4242, oracle_nominal(vs), types, f32(0.8), f32(1.2), f32(0.2),
                                  rg_halfwidth=f32(0.02)))
    np.testing.assert_allclose(got, ref, rtol=2 ** -23, atol=1e-12)
    assert np.abs(got[:, I.P_RG:I.P_RG + 3]).max() > 0.015
    # the fleet steps on the general path and matches the oracle
    sim.reset()
    sim.set_procedural_actions(11, 10)
    s0 = sim.get_state().double().cpu().numpy()
    sim.step(200)
    st = sim.get_state().double().cpu().numpy()
    sim.close()
    cmds = np.stack([np.stack([O.commands(11, e, sg, vs[types[e]].n_thr) for e in range(n)])
                     for sg in range(20)])
    out = O.rollout(got, oracle_geo(vs), types, s0, cmds, 10, 200, h=H)
    assert rel_err(st, out).max() <= TOL_ROLLOUT
