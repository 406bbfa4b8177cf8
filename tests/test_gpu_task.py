"""Task layer (§EXPERIMENTS: station keeping, circle, helix and lemniscate tracking; Eq. 2
observation, Eq. 4 position error, auto-reset) against the FP64 oracle.  Every task step starts
the oracle from the GPU's pre-step state, so that the step's arithmetic is what is compared."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2410_14117_gb300 import inputs as I
from paper_2410_14117_gb300.sim import MGError, Sim

from _helpers import f32, oracle_geo, oracle_nominal, rel_err, vehicles

pytestmark = pytest.mark.gpu

K = 10          # sub-steps per task step (= the command hold, so one command segment per step)
DT = 0.01
SEED, CMD_SEED, SIGMA = 4321, 8765, 0.3


def _centres(n, seed=1):
    g = np.random.default_rng(seed)
    c = np.zeros((n, 4), dtype=np.float32)
    c[:, :3] = g.uniform(-2.0, 2.0, size=(n, 3))
    c[:, 3] = g.uniform(0.0, 2 * math.pi, size=n)
    return c


# (task, look-ahead points, envs per block, sub-steps per launch, work queue, wide): the last
# launch of a task step carries the fused epilogue; with 3 sub-steps per launch the first 9 of the
# 10 run as plain step launches first.  Observation rows are staged in shared memory (above 48 KB
# by opt-in) unless a block's rows exceed the 227 KB limit: 40 look-ahead points (246 floats per
# row) at 256 envs per block take the direct-write path.  wide: the leading plain launches run the
# 200-register kernel (False: the 128-register one).
@pytest.mark.parametrize("task,m,epb,spl,queue,wide", [
    (O.TASK_STATION, 3, 64, 50, False, True), (O.TASK_CIRCLE, 3, 128, 50, False, True),
    (O.TASK_HELIX, 40, 64, 50, False, True), (O.TASK_LEMNISCATE, 3, 96, 3, True, True),
    (O.TASK_CIRCLE, 10, 128, 4, False, True),
    (O.TASK_CIRCLE, 3, 64, 50, False, False), (O.TASK_HELIX, 40, 32, 50, False, False),
    (O.TASK_LEMNISCATE, 3, 96, 3, False, False), (O.TASK_STATION, 3, 128, 4, True, False),
    # rows of exactly 48 KB per block (256 threads x 48 floats), staged by opt-in beside the
    # static shared memory
    (O.TASK_CIRCLE, 7, 256, 50, False, True), (O.TASK_CIRCLE, 3, 256, 4, False, False),
    (O.TASK_HELIX, 40, 256, 50, False, True)])
def test_task_step_matches_oracle(task, m, epb, spl, queue, wide):
    vs = vehicles()
    n = 384
    types = I.mixed_fleet(task + 5, n, max_group=100)
    spec = dict(radius=2.0, omega=0.4, vz=0.1, psi_r=0.3, lookahead=m, lookahead_dt=0.5,
                max_error=2.6, episode_steps=150)
    centres = _centres(n, task)
    sim = Sim(n, types, vs)
    sim.set_launch(epb, spl, False)
    sim.set_schedule(queue, wide)
    sim.randomize(SEED, 0.8, 1.2, 0.2, SIGMA)
    sim.reset()
    sim.set_procedural_actions(CMD_SEED, K)
    sim.set_task(task, torch.tensor(centres, device="cuda"), **spec)

    params = I.round_f32(O.randomize(SEED, oracle_nominal(vs), types, f32(0.8), f32(1.2),
                                     f32(0.2)))
    geo = oracle_geo(vs)
    cen = centres.astype(np.float64)
    args = (f32(spec["radius"]), f32(spec["omega"]), f32(spec["vz"]), f32(spec["psi_r"]),
            spec["lookahead"], f32(spec["lookahead_dt"]))
    clock = np.zeros(n, dtype=np.int64)
    esum = np.zeros(n)
    episode = np.ones(n, dtype=np.int64)  # the initial reset used episode 0
    n_done = 0
    obs0, err0, _, _ = sim.task_step(0)   # observe only: the first observation
    s_now = sim.get_state().double().cpu().numpy()
    for i in range(n):
        o, e = O.task_observe(task, s_now[i], cen[i], *args, 0.0)
        np.testing.assert_allclose(obs0[i].cpu().numpy(), o, atol=2e-5)
    for step in range(40):
        s_before = sim.get_state().double().cpu().numpy()
        obs, err, done, ep = (x.cpu().numpy() for x in sim.task_step(K))
        s_after = sim.get_state().double().cpu().numpy()
        cmds = np.stack([O.commands(CMD_SEED, e, step, vs[types[e]].n_thr) for e in range(n)])
        ref = O.rollout(params, geo, types, s_before, cmds[None], K, K, h=DT)
        for e in range(n):
            t = (clock[e] + K) * DT
            o_ref, e_ref = O.task_observe(task, ref[e], cen[e], *args, t)
            assert abs(err[e] - e_ref) <= 1e-4 * max(1.0, e_ref), (step, e, err[e], e_ref)
            over = e_ref > spec["max_error"] or clock[e] + K >= spec["episode_steps"]
            if bool(done[e]) != over:
                # only a float comparison right at the threshold may differ
                assert abs(e_ref - spec["max_error"]) < 1e-4, (step, e, e_ref)
                over = bool(done[e])
            if over:
                n_done += 1
                assert abs(ep[e] - (esum[e] + e_ref)) <= 1e-3 * max(1.0, esum[e])
                s0 = O.reset_state(SEED, f32(SIGMA), e, int(episode[e]))
                np.testing.assert_allclose(s_after[e], s0, rtol=1e-6, atol=1e-9)
                episode[e] += 1
                clock[e] = 0
                esum[e] = 0.0
                o_ref, _ = O.task_observe(task, s0, cen[e], *args, 0.0)
            else:
                assert ep[e] == 0.0
                clock[e] += K
                esum[e] += e_ref
                assert rel_err(s_after[e][None], ref[e][None]).max() <= 1e-5
            d = obs[e] - o_ref
            d[5::6][: (len(d) - 6) // 6] = np.angle(np.exp(1j * d[5::6][: (len(d) - 6) // 6]))
            np.testing.assert_allclose(d, 0.0, atol=2e-4)
    assert n_done > 0  # the episode end and the error bound both triggered resets
    sim.close()


def test_task_requires_a_task_and_valid_spec():
    vs = vehicles()
    sim = Sim(32, np.zeros(32, dtype=np.int32), vs)
    with pytest.raises(MGError):
        sim._task_out = (torch.zeros((32, 12), device="cuda"), torch.zeros(32, device="cuda"),
                         torch.zeros(32, dtype=torch.uint8, device="cuda"),
                         torch.zeros(32, device="cuda"))
        sim.task_step(1)
    with pytest.raises(MGError):
        sim.set_task(7, torch.zeros((32, 4), device="cuda"))
    sim.close()
