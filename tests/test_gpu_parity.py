"""CUDA path (libmg.so through the C ABI) against the FP64 oracle, element by element, on the
same seeded inputs.  Bars: integer work (Philox) bit-exact; one sub-step <= 1e-5 and 500
sub-steps <= 1e-4 per-block relative error; |q| within 1e-6 of 1 after every sub-step."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2410_14117_gb300 import inputs as I
from paper_2410_14117_gb300.sim import MGError, Sim, philox4x32_10

from _helpers import (TOL_QNORM, TOL_ROLLOUT, TOL_STEP, f32, oracle_geo, oracle_nominal,
                      rel_err, vehicles)

pytestmark = pytest.mark.gpu

H = 0.01


def make_sim(types, vs=None, epb=128, spl=50, graph=True, queue=True, wide=True):
    vs = vs or vehicles()
    sim = Sim(len(types), types, vs)
    sim.set_launch(epb, spl, graph)
    sim.set_schedule(queue, wide)
    return sim


def gpu_state(sim):
    return sim.get_state().cpu().numpy().astype(np.float64)


def oracle_types_geo(types, vs):
    return np.asarray(types, dtype=np.int32), oracle_geo(vs)


# ----------------------------------------------------------------------------- RNG (integer)

def test_philox_bit_exact_known_answers_and_random():
    kat = np.array([[0, 0, 0, 0, 0, 0], [0xffffffff] * 6,
                    [0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344, 0xa4093822, 0x299f31d0]],
                   dtype=np.uint64).astype(np.uint32)
    want = np.array([[0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8],
                     [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd],
                     [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]], dtype=np.uint32)
    np.testing.assert_array_equal(philox4x32_10(kat[:, :4], kat[:, 4:]), want)
    g = np.random.default_rng(1)
    ctr = g.integers(0, 2**32, size=(5000, 4), dtype=np.uint64).astype(np.uint32)
    key = g.integers(0, 2**32, size=(5000, 2), dtype=np.uint64).astype(np.uint32)
    got = philox4x32_10(ctr, key)
    ref = np.array([O.philox4x32_10(c, k) for c, k in zip(ctr[:500], key[:500])])
    np.testing.assert_array_equal(got[:500], ref)


# ----------------------------------------------------------------------------- randomiser

@pytest.mark.parametrize("offset", [0, 12345])
def test_randomize_matches_oracle(offset):
    vs = vehicles()
    types = I.mixed_fleet(3, 5000, max_group=700)
    sim = make_sim(types, vs)
    sim.set_env_id_offset(offset)
    lo, hi, sc = f32(0.8), f32(1.2), f32(0.2)
    sim.randomize(1234, 0.8, 1.2, 0.2, 0.3)
    got = sim.get_params().cpu().numpy().astype(np.float64)
    ref = O.randomize(1234, oracle_nominal(vs), types, lo, hi, sc, gid0=offset)
    # The device draws in FP64 and stores FP32: equal to the oracle's value rounded to FP32, up
    # to the last FP64 bit of the arithmetic before rounding.
    np.testing.assert_allclose(got, ref, rtol=2.0 ** -24 * 1.01, atol=1e-30)
    sim.close()


def test_reset_draw_matches_oracle():
    types = np.zeros(3000, dtype=np.int32)
    sim = make_sim(types)
    sim.randomize(77, 0.8, 1.2, 0.2, 0.3)
    sim.reset()
    sim.reset(torch.tensor(np.arange(3000) % 3 == 0, dtype=torch.uint8, device="cuda"))
    got = gpu_state(sim)
    for e in range(0, 3000, 7):
        ep = 1 if e % 3 == 0 else 0
        ref = O.reset_state(77, f32(0.3), e, ep)
        np.testing.assert_allclose(got[e], ref, rtol=1e-6, atol=1e-9)
    sim.close()


# ----------------------------------------------------------------------------- one sub-step

def _teacher_forced(types, vs, params, states, cmds, flags=0, epb=128):
    sim = make_sim(types, vs, epb=epb)
    sim.set_model_flags(flags)
    sim.set_params(torch.tensor(params, dtype=torch.float32, device="cuda"))
    sim.set_state(torch.tensor(states, dtype=torch.float32, device="cuda"))
    sim.set_actions(torch.tensor(cmds[None], dtype=torch.float32, device="cuda"), 1)
    sim.step(1)
    got = gpu_state(sim)
    sim.close()
    t, geo = oracle_types_geo(types, vs)
    ref = O.rollout(params, geo, t, states, cmds[None], 1, 1, h=H, flags=flags)
    return got, ref


@pytest.mark.parametrize("flags", [0, 1])
def test_one_substep_randomised_with_current(flags):
    vs = vehicles()
    n = 4096
    types = I.mixed_fleet(11, n, max_group=300)
    nt = np.array([vs[t].n_thr for t in types])
    params = I.perturbed_params(5, oracle_nominal(vs)[types], n)
    states = I.random_states(6, n, nt)
    cmds = I.commands(7, 1, n, nt)[0].astype(np.float64)
    got, ref = _teacher_forced(types, vs, params, states, cmds, flags)
    err = rel_err(got, ref)
    assert err.max() <= TOL_STEP, err.max(axis=0)


def test_one_substep_off_centre_gravity_general_path():
    vs = vehicles()
    n = 2048
    types = np.zeros(n, dtype=np.int32)
    params = I.perturbed_params(8, oracle_nominal(vs)[types], n)
    g = np.random.default_rng(9)
    params[:, I.P_RG:I.P_RG + 3] = I.round_f32(g.uniform(-0.03, 0.03, (n, 3)))
    states = I.random_states(10, n, 6)
    cmds = I.commands(11, 1, n, 6)[0].astype(np.float64)
    got, ref = _teacher_forced(types, vs, params, states, cmds)
    err = rel_err(got, ref)
    assert err.max() <= TOL_STEP, err.max(axis=0)


# ----------------------------------------------------------------------------- rollouts

def _rollout_compare(types, vs, params, s0, cmds, hold, n_steps, epb=128, spl=50, graph=True,
                     check_every=50):
    """Step the GPU n_steps (recording the trajectory) and the oracle alike; return the
    per-block errors at every check point and the quaternion-norm deviation."""
    sim = make_sim(types, vs, epb=epb, spl=spl, graph=graph)
    sim.set_params(torch.tensor(params, dtype=torch.float32, device="cuda"))
    sim.set_state(torch.tensor(s0, dtype=torch.float32, device="cuda"))
    sim.set_actions(torch.tensor(cmds, dtype=torch.float32, device="cuda"), hold)
    traj = sim.step_record(n_steps).cpu().numpy().astype(np.float64)  # [T, 13, n]
    final = gpu_state(sim)
    sim.close()
    t, geo = oracle_types_geo(types, vs)
    ref_final, ref_traj = O.rollout(params, geo, t, s0, cmds.astype(np.float64), hold, n_steps,
                                    h=H, record=True)
    errs = []
    for j in range(check_every - 1, n_steps, check_every):
        g = np.zeros_like(ref_traj[j])
        g[:, :13] = traj[j].T
        r = ref_traj[j].copy()
        r[:, 13:] = 0.0
        errs.append(rel_err(g, r).max())
    qn = np.abs(np.linalg.norm(traj[:, 3:7, :], axis=1) - 1.0).max()
    return np.array(errs), rel_err(final, ref_final), qn


def test_small_fleet_500_substeps_nominal():
    """1,024 BlueROV2, nominal parameters, no current, commands U[-1,1] held 10 sub-steps,
    nu0 ~ N(0, 0.3), identity attitude, 500 sub-steps of 0.01 s."""
    vs = vehicles()
    n = 1024
    types = np.zeros(n, dtype=np.int32)
    params = np.broadcast_to(oracle_nominal(vs)[0], (n, I.NPARAM)).copy()
    s0 = I.initial_states(21, n)
    cmds = I.commands(5678, 50, n, 6)
    errs, final, qn = _rollout_compare(types, vs, params, s0, cmds, 10, 500)
    assert errs.max() <= TOL_ROLLOUT and final.max() <= TOL_ROLLOUT, (errs, final.max(axis=0))
    assert qn <= TOL_QNORM


def test_randomised_fleet_with_current_500_substeps():
    """Domain-randomised parameters and NED current drawn on the device, oracle drawing its own
    from the same counter-based generator."""
    vs = vehicles()
    n = 4096
    types = np.zeros(n, dtype=np.int32)
    sim = make_sim(types, vs)
    sim.randomize(1234, 0.8, 1.2, 0.2, 0.3)
    sim.reset()
    cmds = I.commands(5678, 50, n, 6)
    sim.set_actions(torch.tensor(cmds, device="cuda"), 10)
    sim.step(500)
    got = gpu_state(sim)
    sim.close()
    params = I.round_f32(O.randomize(1234, oracle_nominal(vs), types, f32(0.8), f32(1.2),
                                     f32(0.2)))
    s0 = np.stack([I.round_f32(O.reset_state(1234, f32(0.3), e, 0)) for e in range(n)])
    ref = O.rollout(params, oracle_geo(vs), types, s0, cmds.astype(np.float64), 10, 500, h=H)
    err = rel_err(got, ref)
    assert err.max() <= TOL_ROLLOUT, err.max(axis=0)


@pytest.mark.parametrize("n,epb,spl,graph", [(1, 32, 50, True), (31, 32, 7, False),
                                             (33, 64, 1, False), (257, 96, 13, True),
                                             (1000, 256, 500, True)])
def test_ragged_sizes_and_launch_shapes(n, epb, spl, graph):
    vs = vehicles()
    types = I.mixed_fleet(n, n, max_group=40)
    nt = np.array([vs[t].n_thr for t in types])
    params = I.perturbed_params(n + 1, oracle_nominal(vs)[types], n)
    s0 = I.random_states(n + 2, n, nt, nu_sigma=0.3)
    cmds = I.commands(n + 3, 20, n, nt)
    errs, final, qn = _rollout_compare(types, vs, params, s0, cmds, 10, 200, epb=epb, spl=spl,
                                       graph=graph)
    assert errs.max() <= TOL_ROLLOUT and final.max() <= TOL_ROLLOUT
    assert qn <= TOL_QNORM


@pytest.mark.parametrize("general", [False, True])
def test_schedule_and_launch_shape_do_not_change_results(general):
    """Same arithmetic per env whatever the schedule (work queue or static grid), register budget
    (128 or 200), block size, chunking or graph replay: bitwise equal final states."""
    vs = vehicles()
    n = 3000
    types = I.mixed_fleet(4, n, max_group=500)
    params = None
    if general:
        params = I.perturbed_params(3, oracle_nominal(vs)[types], n)
        params[:, I.P_RG:I.P_RG + 3] = I.round_f32(
            np.random.default_rng(2).uniform(-0.02, 0.02, (n, 3)))
    out = []
    for epb, spl, graph, queue, wide in [(128, 50, True, True, True), (64, 1, False, False, False),
                                         (256, 17, True, False, True), (32, 300, False, True, False),
                                         (96, 7, False, True, True), (128, 1, True, True, True),
                                         (32, 300, True, False, True), (64, 50, False, False, False)]:
        sim = make_sim(types, vs, epb=epb, spl=spl, graph=graph, queue=queue, wide=wide)
        if general:
            sim.set_params(torch.tensor(params, dtype=torch.float32, device="cuda"))
            sim.set_state(torch.tensor(I.random_states(5, n, [vs[t].n_thr for t in types]),
                                       dtype=torch.float32, device="cuda"))
        else:
            sim.randomize(9, 0.8, 1.2, 0.2, 0.3)
            sim.reset()
        sim.set_procedural_actions(99, 10)
        sim.step(150)
        sim.step(150)
        assert sim.sync() == 0
        out.append(gpu_state(sim))
        sim.close()
    for o in out[1:]:
        np.testing.assert_array_equal(o, out[0])


@pytest.mark.parametrize("queue", [False, True])
def test_graph_replay_follows_the_device_cursor(queue):
    """The action cursor lives on the device, so one cached graph per k replays at any cursor:
    many short graph-replayed steps (crossing hold and buffer boundaries, and a re-set of the
    same-shaped actions in mid-run) equal one long direct step sequence bit for bit."""
    vs = vehicles()
    n = 1500
    types = I.mixed_fleet(21, n, max_group=400)
    nt = [vs[t].n_thr for t in types]
    a1 = torch.tensor(I.commands(31, 12, n, nt), device="cuda")
    a2 = torch.tensor(I.commands(32, 12, n, nt), device="cuda")
    out = []
    for graph in (False, True):
        sim = make_sim(types, vs, spl=5, graph=graph, queue=queue)
        sim.randomize(13, 0.8, 1.2, 0.2, 0.3)
        sim.reset()
        sim.set_actions(a1, 7)
        if graph:
            for _ in range(19):
                sim.step(7)
            sim.step(3)
            sim.step(3)
        else:
            sim.step(139)
        sim.set_actions(a2, 7)   # same shape: the cached graphs stay, the cursor rewinds
        if graph:
            for _ in range(11):
                sim.step(7)
        else:
            sim.step(77)
        sim.set_procedural_actions(5, 4)
        if graph:
            for _ in range(9):
                sim.step(3)
        else:
            sim.step(27)
        assert sim.sync() == 0
        out.append(gpu_state(sim))
        sim.close()
    np.testing.assert_array_equal(out[1], out[0])


def test_borrowed_actions_equal_copied_actions():
    vs = vehicles()
    n = 2000
    types = I.mixed_fleet(8, n, max_group=300)
    cmds = torch.tensor(I.commands(9, 30, n, [vs[t].n_thr for t in types]), device="cuda")
    out = []
    for borrowed in (False, True):
        sim = make_sim(types, vs, spl=25, queue=borrowed)
        sim.randomize(3, 0.8, 1.2, 0.2, 0.3)
        sim.reset()
        if borrowed:
            sim.set_actions_borrowed(cmds, 10)
        else:
            sim.set_actions(cmds, 10)
        sim.step(170)
        sim.step(130)
        out.append(gpu_state(sim))
        sim.close()
    np.testing.assert_array_equal(out[0], out[1])
    sim = make_sim(types, vs)
    with pytest.raises((ValueError, MGError)):
        sim.set_actions_borrowed(cmds.cpu(), 10)
    sim.close()


def test_procedural_commands_match_oracle():
    vs = vehicles()
    n = 512
    types = I.mixed_fleet(12, n, max_group=100)
    sim = make_sim(types, vs)
    sim.randomize(5, 0.8, 1.2, 0.2, 0.3)
    sim.reset()
    sim.set_procedural_actions(4242, 10)
    sim.step(200)
    got = gpu_state(sim)
    sim.close()
    params = I.round_f32(O.randomize(5, oracle_nominal(vs), types, f32(0.8), f32(1.2), f32(0.2)))
    s0 = np.stack([I.round_f32(O.reset_state(5, f32(0.3), e, 0)) for e in range(n)])
    cmds = np.stack([np.stack([O.commands(4242, e, sg, vs[types[e]].n_thr) for e in range(n)])
                     for sg in range(20)])
    ref = O.rollout(params, oracle_geo(vs), types, s0, cmds, 10, 200, h=H)
    err = rel_err(got, ref)
    assert err.max() <= TOL_ROLLOUT, err.max(axis=0)


def test_literal_frame_reading_short_horizon():
    """The literal (statically unstable) reading of the experiment's body-frame vectors runs
    through the same kernels; over 100 sub-steps errors stay within the rollout bar."""
    vs = vehicles("literal")
    n = 512
    types = np.zeros(n, dtype=np.int32)
    params = np.broadcast_to(oracle_nominal(vs)[0], (n, I.NPARAM)).copy()
    s0 = I.initial_states(3, n)
    cmds = I.commands(4, 10, n, 6)
    errs, final, _ = _rollout_compare(types, vs, params, s0, cmds, 10, 100)
    assert final.max() <= TOL_ROLLOUT


# ----------------------------------------------------------------------------- failure paths

def test_nonfinite_is_flagged_and_confined():
    vs = vehicles()
    n = 64
    types = np.zeros(n, dtype=np.int32)
    params = np.broadcast_to(oracle_nominal(vs)[0], (n, I.NPARAM)).copy()
    params[17, I.P_DQ] = np.nan
    s0 = I.initial_states(1, n)
    sim = make_sim(types, vs)
    sim.set_params(torch.tensor(params, dtype=torch.float32, device="cuda"))
    sim.set_state(torch.tensor(s0, dtype=torch.float32, device="cuda"))
    sim.step(20)
    assert sim.sync() == 1
    mask = sim.nonfinite_mask().cpu().numpy()
    assert mask[17] == 1 and mask.sum() == 1
    got = gpu_state(sim)
    ok = np.arange(n) != 17
    ref = O.rollout(np.where(np.isnan(params), 0.0, params)[ok], oracle_geo(vs), types[ok],
                    s0[ok], np.zeros((1, ok.sum(), 8)), 1, 20, h=H)
    assert rel_err(got[ok], ref).max() <= TOL_ROLLOUT
    sim.reset(torch.tensor(~ok, dtype=torch.uint8, device="cuda"))
    assert sim.sync() == 0
    sim.close()


def test_not_spd_reported():
    vs = vehicles()
    n = 40
    types = np.zeros(n, dtype=np.int32)
    params = np.broadcast_to(oracle_nominal(vs)[0], (n, I.NPARAM)).copy()
    params[3, I.P_M] = -30.0
    sim = make_sim(types, vs)
    with pytest.raises(MGError) as ei:
        sim.set_params(torch.tensor(params, dtype=torch.float32, device="cuda"))
    assert ei.value.code == "MG_ENOTSPD"
    sim.close()


def test_async_randomize_equals_sync_and_reports_not_spd_at_sync():
    """MG_RANDOMIZE_ASYNC draws the same parameters without waiting; a mass matrix that is not
    positive definite then surfaces at mg_sync; fleets whose mass matrix may be full reject it."""
    import dataclasses
    vs = vehicles()
    n = 3000
    types = I.mixed_fleet(17, n, max_group=400)
    out = []
    for wait in (True, False):
        sim = make_sim(types, vs)
        sim.randomize(55, 0.8, 1.2, 0.2, 0.3, wait=wait)
        sim.reset()
        sim.set_procedural_actions(56, 10)
        sim.step(100)
        assert sim.sync() == 0
        out.append((sim.get_params().cpu(), gpu_state(sim)))
        sim.close()
    assert torch.equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    # surge added mass -11 kg against 11.5 kg: the nominal mass matrix is positive definite,
    # but many draws (m x U[0.8,1.2] + M_A x U[0.8,1.2]) are not; accepted without waiting,
    # reported by sync
    bad = [dataclasses.replace(v, params=v.params.copy()) for v in vs]
    bad[0].params[I.P_MA] = -11.0
    sim = Sim(64, np.zeros(64, np.int32), bad)
    sim.randomize(1, 0.8, 1.2, 0.2, 0.3, wait=False)
    with pytest.raises(MGError) as ei:
        sim.sync()
    assert ei.value.code == "MG_ENOTSPD"
    sim.close()
    sim = make_sim(types, vs)
    with pytest.raises(MGError) as ei:
        sim.randomize(1, 0.8, 1.2, 0.2, 0.3, rg_halfwidth=0.01, wait=False)
    assert ei.value.code == "MG_EINVAL"
    sim.close()


def test_invalid_arguments_rejected_on_host():
    vs = vehicles()
    sim = make_sim(np.zeros(10, dtype=np.int32), vs)
    for fn, args in [(sim.step, (0,)), (sim.set_launch, (16, 1, True)),
                     (sim.set_launch, (128, 0, True)), (sim.set_timestep, (-1.0,)),
                     (sim.randomize, (1, 1.2, 0.8))]:
        with pytest.raises(MGError) as ei:
            fn(*args)
        assert ei.value.code == "MG_EINVAL"
    bad = [(sim.set_actions, (None, 0)), (sim.set_procedural_actions, (1, 0)),
           (sim.set_schedule, (True, True, 65)), (sim.step_record, (0,)),
           (sim.randomize, (1, 0.8, 1.2, -0.1)), (sim.randomize, (1, 0.8, 1.2, 0.2, -0.3)),
           (sim.randomize, (1, 0.0, 1.2)), (sim.set_timestep, (2.0,))]
    for fn, args in bad:
        with pytest.raises(MGError) as ei:
            fn(*args)
        assert ei.value.code == "MG_EINVAL", (fn, args)
    r = sim.get_params()
    with pytest.raises(MGError):
        sim.randomize(1, 0.8, 1.2, 0.2, 0.3, rg_halfwidth=-0.01)
    torch.testing.assert_close(sim.get_params(), r, rtol=0, atol=0)  # nothing changed
    with pytest.raises(MGError):
        sim.set_task(0, torch.zeros((10, 4), device="cuda"), lookahead=65)
    with pytest.raises(MGError):
        Sim(10, np.full(10, 5), vs)
    with pytest.raises((MGError, ValueError)):
        Sim(0, np.zeros(0, dtype=np.int32), vs)
    sim.close()
