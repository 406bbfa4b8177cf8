"""Parity at the benchmark's full sizes, in the launch configurations the benchmark times, on
sampled envs the oracle computes one by one: the 65,536-env headline fleet (work-queue kernel,
200-register cap, 8 warps/SM, chunk 100, the unpadded 6-float throttle schedule read in place,
CUDA graph) over a whole 1,000 sub-step episode, parameters drawn in the background and
installed as the benchmark does them; the 262,144-env mixed fleet over 500 sub-steps and the
1,048,576-env top of the size sweep (each also on the 200-register static grid the autotuner picks
for them)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2410_14117_gb300 import inputs as I
from paper_2410_14117_gb300.autotune import LaunchConfig
from paper_2410_14117_gb300.sim import Sim

from _helpers import TOL_ROLLOUT, f32, oracle_geo, oracle_nominal, rel_err, vehicles

pytestmark = pytest.mark.gpu

H = 0.01


def _sample(n, k, seed):
    g = np.random.default_rng(seed)
    pick = set(g.choice(n, size=k, replace=False).tolist()) | {0, 31, 32, n - 33, n - 1}
    return np.array(sorted(pick))


def _oracle_rollout(vs, types, sample, seed, cmds, hold, steps):
    """The sampled envs' randomised parameters, start states and commands, drawn by the oracle
    from the same counter-based generator (keyed by each env's global id), then rolled out."""
    nominal = oracle_nominal(vs)
    par = np.concatenate([O.randomize(seed, nominal, types[e:e + 1], f32(0.8), f32(1.2),
                                      f32(0.2), gid0=int(e)) for e in sample])
    par = I.round_f32(par)
    s0 = np.stack([I.round_f32(O.reset_state(seed, f32(0.3), int(e), 0)) for e in sample])
    return O.rollout(par, oracle_geo(vs), types[sample], s0,
                     cmds[:, sample].astype(np.float64), hold, steps, h=H)


def test_headline_fleet_sampled_matches_oracle():
    vs = vehicles()
    n, hold = 65536, 10
    types = np.zeros(n, dtype=np.int32)
    sim = Sim(n, types, vs)
    LaunchConfig("queue", 128, 100, True, 8).apply(sim)
    sim.set_action_width(6)  # the benchmark's unpadded schedule
    # the parameters reach the fleet as in the benchmark: drawn in the background, installed
    sim.randomize_prefetch(1234, 0.8, 1.2, 0.2)
    sim.randomize(1234, 0.8, 1.2, 0.2, 0.3, wait=False)
    sim.reset()
    cmds = I.commands(5678, 100, n, 6)
    acts = torch.tensor(np.ascontiguousarray(cmds[:, :, :6]), device="cuda")
    sim.set_actions_borrowed(acts, hold)
    sample = _sample(n, 600, 3)
    sim.step(500)
    mid = sim.get_state().double().cpu().numpy()[sample]
    sim.step(500)
    end = sim.get_state().double().cpu().numpy()[sample]
    assert sim.sync() == 0
    sim.close()
    ref_mid = _oracle_rollout(vs, types, sample, 1234, cmds, hold, 500)
    err_mid = rel_err(mid, ref_mid)
    ref_end = _oracle_rollout(vs, types, sample, 1234, cmds, hold, 1000)
    err_end = rel_err(end, ref_end)
    msg = (f"max per-block error after 500 sub-steps {err_mid.max():.3e} "
           f"(p, q, v, w, n: {np.array2string(err_mid.max(axis=0), precision=3)}), after 1,000 "
           f"{err_end.max():.3e} ({np.array2string(err_end.max(axis=0), precision=3)})")
    print(msg)
    assert err_mid.max() <= TOL_ROLLOUT, msg
    # the whole episode is held to the same bar as 500 sub-steps
    assert err_end.max() <= TOL_ROLLOUT, msg


@pytest.mark.parametrize("launch", [LaunchConfig("queue", 128, 50, True, 12),
                                    LaunchConfig("static", 32, 1000, True)])
def test_mixed_fleet_262144_sampled_matches_oracle(launch):
    vs = vehicles()
    n, hold = 262144, 10
    types = I.mixed_fleet(3, n)
    sim = Sim(n, types, vs)
    launch.apply(sim)
    sim.randomize(4321, 0.8, 1.2, 0.2, 0.3)
    sim.reset()
    nt = np.array([vs[t].n_thr for t in types])
    cmds = I.commands(8765, 50, n, nt)
    sim.set_actions(torch.tensor(cmds, device="cuda"), hold)
    sim.step(500)
    sample = _sample(n, 400, 4)
    got = sim.get_state().double().cpu().numpy()[sample]
    assert sim.sync() == 0
    sim.close()
    ref = _oracle_rollout(vs, types, sample, 4321, cmds, hold, 500)
    err = rel_err(got, ref)
    assert err.max() <= TOL_ROLLOUT, err.max(axis=0)


@pytest.mark.parametrize("launch", [LaunchConfig("static", 128, 200),
                                    LaunchConfig("static", 64, 1000, True)])
def test_largest_sweep_fleet_sampled_matches_oracle(launch):
    """1,048,576 envs (the top of the fleet-size sweep), static grid, 200 sub-steps."""
    vs = vehicles()
    n, hold = 1 << 20, 10
    types = np.zeros(n, dtype=np.int32)
    sim = Sim(n, types, vs)
    launch.apply(sim)
    sim.randomize(99, 0.8, 1.2, 0.2, 0.3)
    sim.reset()
    cmds = I.commands(98, 20, n, 6)
    sim.set_actions(torch.tensor(cmds, device="cuda"), hold)
    sim.step(200)
    sample = _sample(n, 300, 5)
    got = sim.get_state().double().cpu().numpy()[sample]
    assert sim.sync() == 0
    sim.close()
    ref = _oracle_rollout(vs, types, sample, 99, cmds, hold, 200)
    err = rel_err(got, ref)
    assert err.max() <= TOL_ROLLOUT, err.max(axis=0)
