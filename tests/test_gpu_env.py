"""Gym-style environment (MarineEnv) over the fused task step: each env step gives the bits of
the task step it wraps, its observations and errors match the FP64 oracle from the GPU's
pre-step state, episodes end and restart inside the step, and shapes and arguments are
checked."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2410_14117_gb300 import inputs as I
from paper_2410_14117_gb300.env import TASKS, MarineEnv
from paper_2410_14117_gb300.sim import Sim

from _helpers import f32, oracle_geo, rel_err, vehicles

pytestmark = pytest.mark.gpu

SPEC = dict(radius=2.0, omega=0.3, vz=0.1, psi_r=0.0, lookahead=4, lookahead_dt=0.5,
            max_error=3.0, episode_steps=1000)


def _actions(step, n, nt, scale=1.3):
    g = torch.Generator(device="cpu").manual_seed(1000 + step)
    return ((torch.rand((n, nt), generator=g) * 2 - 1) * scale).cuda()


# k = 60 runs its first 50 sub-steps as a graph-replayed mg_step on the library's schedule
@pytest.mark.parametrize("mixed,k", [(False, 10), (True, 10), (False, 60)])
def test_env_step_equals_the_task_step_it_wraps(mixed, k):
    n, seed = 700, 3
    types = I.mixed_fleet(8, n, max_group=90) if mixed else np.full(n, 1, dtype=np.int32)
    env = MarineEnv(n, task="helix", vehicle=types if mixed else 1, sub_steps=k, seed=seed,
                    nu0_sigma=0.2)
    vs = I.fleet_vehicles()
    sim = Sim(n, types, vs)
    sim.randomize(seed, 0.8, 1.2, 0.2, 0.2)
    sim.reset()
    sim.set_task(TASKS["helix"], env.centres.clone(), **SPEC)
    act = torch.zeros((1, n, 8), device="cuda")
    for step in range(15):
        a = _actions(step, n, 8)
        obs, rew, done, info = env.step(a)
        act[0] = a.clamp(-1, 1)
        sim.set_actions_borrowed(act, k)
        o2, e2, d2, ep2 = sim.task_step(k)
        assert torch.equal(obs, o2) and torch.equal(rew, -e2)
        assert torch.equal(done, d2.bool()) and torch.equal(info["episode_error"], ep2)
    assert torch.equal(env.sim.get_state(), sim.get_state())
    env.close()
    sim.close()


@pytest.mark.parametrize("task,vehicle", [("station", 0), ("circle", 1), ("lemniscate", 0)])
def test_env_matches_oracle(task, vehicle):
    """Three env steps from reset: the oracle integrates each env from the GPU's pre-step state
    with the held (clamped) throttles and observes it at the step's end (Eq. 2, Eq. 4)."""
    n, k = 256, 10
    env = MarineEnv(n, task=task, vehicle=vehicle, sub_steps=k, seed=11, nu0_sigma=0.3)
    nt = env.n_thr
    vs = vehicles()
    geo = oracle_geo(vs)
    params = env.sim.get_params().double().cpu().numpy()
    types = np.full(n, vehicle, dtype=np.int32)
    cen = env.centres.double().cpu().numpy()
    args = (f32(SPEC["radius"]), f32(SPEC["omega"]), f32(SPEC["vz"]), f32(SPEC["psi_r"]),
            SPEC["lookahead"], f32(SPEC["lookahead_dt"]))
    obs0 = env.reset().cpu().numpy()
    s = env.sim.get_state().double().cpu().numpy()
    for e in range(n):
        o, _ = O.task_observe(TASKS[task], s[e], cen[e], *args, 0.0)
        np.testing.assert_allclose(obs0[e], o, atol=2e-5)
    for step in range(3):
        a = _actions(step, n, nt)
        s_before = env.sim.get_state().double().cpu().numpy()
        obs, rew, done, _ = (x.cpu().numpy() if torch.is_tensor(x) else x for x in env.step(a))
        assert not done.any()
        cmd = np.zeros((1, n, 8))
        cmd[0, :, :nt] = a.clamp(-1, 1).double().cpu().numpy()
        ref = O.rollout(params, geo, types, s_before, cmd, k, k, h=0.01)
        s_after = env.sim.get_state().double().cpu().numpy()
        assert rel_err(s_after, ref).max() <= 1e-5
        t = (step + 1) * k * 0.01
        for e in range(n):
            o_ref, e_ref = O.task_observe(TASKS[task], ref[e], cen[e], *args, t)
            assert abs(-rew[e] - e_ref) <= 1e-4 * max(1.0, e_ref)
            d = obs[e] - o_ref
            m = (len(d) - 6) // 6
            d[5::6][:m] = np.angle(np.exp(1j * d[5::6][:m]))  # heading error wraps at +-pi
            np.testing.assert_allclose(d, 0.0, atol=2e-4)
    env.close()


def test_env_episodes_end_and_restart_inside_the_step():
    n, k = 300, 10
    env = MarineEnv(n, task="circle", vehicle=1, sub_steps=k, seed=5, max_error=1e6,
                    episode_steps=40)
    zero = torch.zeros((n, 8), device="cuda")
    for step in range(1, 9):
        _, rew, done, info = env.step(zero)
        if step % 4:
            assert not done.any() and not info["episode_error"].any()
        else:
            assert done.all()
            assert (info["episode_error"] > 0).all()
            s = env.sim.get_state().cpu()
            assert not s[:, 0:3].any()  # the new episode starts at the origin
    env.close()


def test_env_shapes_and_arguments():
    env = MarineEnv(64, task="station", vehicle=0, sub_steps=5, seed=1)
    assert env.obs_dim == 12 and env.action_dim == 6 and env.sim.act_w == 6
    obs = env.reset()
    assert tuple(obs.shape) == (64, 12)
    with pytest.raises(ValueError):
        env.step(torch.zeros((64, 8), device="cuda"))
    obs, rew, done, info = env.step(np.zeros((64, 6), dtype=np.float32))
    assert rew.dtype == torch.float32 and done.dtype == torch.bool and rew.is_cuda
    env.close()
    with pytest.raises(ValueError):
        MarineEnv(8, task="orbit")
    with pytest.raises(ValueError):
        MarineEnv(8, sub_steps=0)
    with pytest.raises(ValueError):
        MarineEnv(8, vehicle=[0, 1])
    assert math.isclose(float(TASKS["helix"]), 2.0)


def test_env_step_entry_point_errors_and_switching_back():
    """mg_env_step rejects what it cannot run on the host; after environment steps an ordinary
    action schedule takes over again, with the bits of a sim that never used mg_env_step."""
    import ctypes
    from paper_2410_14117_gb300._lib import MGError, call
    n, k = 128, 10
    env = MarineEnv(n, task="circle", vehicle=1, sub_steps=k, seed=9)
    sim = env.sim
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    obs, rew, ep = env._obs, env._rew, env._ep
    done = env._done
    host = torch.zeros((n, 8))
    for bad_k, acts in ((0, torch.zeros((n, 8), device="cuda")), (k, host)):
        with pytest.raises(MGError) as ei:
            call("mg_env_step", sim._h, bad_k, ptr(acts), ptr(obs), ptr(rew), ptr(done), ptr(ep))
        assert ei.value.code == "MG_EINVAL"
    plain = Sim(n, np.full(n, 1, dtype=np.int32), I.fleet_vehicles())
    with pytest.raises(MGError) as ei:
        call("mg_env_step", plain._h, k, ptr(torch.zeros((n, 8), device="cuda")), ptr(obs),
             ptr(rew), ptr(done), ptr(ep))
    assert ei.value.code == "MG_ESTATE"
    plain.close()
    # two environment steps, then an ordinary schedule on both this sim and a twin
    twin = Sim(n, np.full(n, 1, dtype=np.int32), I.fleet_vehicles())
    twin.randomize(9, 0.8, 1.2, 0.2, 0.0)
    twin.reset()
    twin.set_task(TASKS["circle"], env.centres.clone(), **SPEC)
    tact = torch.zeros((1, n, 8), device="cuda")
    for step in range(2):
        a = _actions(step, n, 8)
        env.step(a)
        tact[0] = a.clamp(-1, 1)
        twin.set_actions_borrowed(tact, k)
        twin.task_step(k)
    cmds = torch.tensor(I.commands(4, 3, n, 8), device="cuda")
    for s_ in (sim, twin):
        s_.set_actions(cmds, 10)
        s_.step(30)
    assert torch.equal(sim.get_state(), twin.get_state())
    env.close()
    twin.close()


def test_env_non_finite_throttles_end_the_episode():
    """A NaN throttle (kept by the clamp) makes that env's state non-finite within the step; the
    step ends its episode and resets it (done, a finite start state at the origin), and the
    other envs carry on untouched."""
    n, k = 256, 10
    env = MarineEnv(n, task="station", vehicle=0, sub_steps=k, seed=4)
    a = torch.zeros((n, 6), device="cuda")
    env.step(a)
    a[7, 2] = float("nan")
    _, rew, done, _ = env.step(a)
    assert bool(done[7]) and int(done.sum()) == 1
    s = env.sim.get_state()
    assert torch.isfinite(s).all() and not s[7, 0:3].any()
    assert torch.isfinite(rew[torch.arange(n, device="cuda") != 7]).all()
    assert env.sim.sync() == 0  # the reset cleared the env's non-finite flag
    # the others advanced exactly as they would have with zero throttles everywhere
    twin = MarineEnv(n, task="station", vehicle=0, sub_steps=k, seed=4)
    twin.step(torch.zeros((n, 6), device="cuda"))
    twin.step(torch.zeros((n, 6), device="cuda"))
    keep = torch.arange(n, device="cuda") != 7
    assert torch.equal(s[keep], twin.sim.get_state()[keep])
    env.close()
    twin.close()
