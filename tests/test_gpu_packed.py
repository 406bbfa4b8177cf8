"""Packed FP32x2 step kernels (two envs per thread, mg_set_packed) against the one-env-per-thread
kernels, bit for bit, and against the FP64 oracle.  A packed FMA is two correctly rounded FMAs,
so the packed kernels must reproduce the scalar kernels' bits for every env, fleet shape, launch
shape and model flag.  The packed form runs on the static grid; with the work-queue schedule the
setting is ignored (those shapes check that the fall-back is seamless)."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2410_14117_gb300 import inputs as I
from paper_2410_14117_gb300._lib import MG_MODEL_NO_CURRENT_ACCEL
from paper_2410_14117_gb300.sim import Sim

from _helpers import TOL_ROLLOUT, f32, oracle_geo, oracle_nominal, rel_err, vehicles

pytestmark = pytest.mark.gpu

H = 0.01
SHAPES = [(128, 50, True, True), (64, 1, False, False), (256, 17, True, False),
          (32, 300, False, True), (96, 7, False, False), (128, 1000, True, False)]


def _tilted(vs):
    """Vertical thrusters tilted 0.1 rad about y: not the vectored layout (dense allocation)."""
    out = []
    for v in vs:
        d = v.d.copy()
        for i in range(4, v.n_thr):
            d[i] = (np.sin(0.1), 0.0, np.cos(0.1))
        out.append(dataclasses.replace(v, d=d))
    return out


def _fleet(kind, n):
    vs = vehicles()
    if kind == "bluerov2":
        return np.zeros(n, np.int32), vs
    if kind == "heavy":
        return np.ones(n, np.int32), vs
    if kind == "mixed":
        return I.mixed_fleet(n + 7, n, max_group=max(1, n // 5)), vs
    return I.mixed_fleet(n + 8, n, max_group=max(1, n // 3)), _tilted(vs)


def _run(types, vs, packed, shape, flags=0, steps=(150, 150), actions=None):
    epb, spl, graph, queue = shape
    sim = Sim(len(types), types, vs)
    sim.set_launch(epb, spl, graph)
    sim.set_schedule(queue)
    sim.set_packed(packed)
    sim.set_model_flags(flags)
    sim.randomize(9, 0.8, 1.2, 0.2, 0.3)
    sim.reset()
    if actions is None:
        sim.set_procedural_actions(99, 10)
    else:
        sim.set_actions(actions, 7)
    for k in steps:
        sim.step(k)
    assert sim.sync() == 0
    out = sim.get_state().cpu().numpy()
    sim.close()
    return out


@pytest.mark.parametrize("kind", ["bluerov2", "heavy", "mixed", "tilted"])
@pytest.mark.parametrize("n", [1, 33, 100, 3000])
def test_packed_equals_scalar_bitwise(kind, n):
    types, vs = _fleet(kind, n)
    ref = _run(types, vs, False, SHAPES[0])
    for shape in SHAPES:
        np.testing.assert_array_equal(_run(types, vs, True, shape), ref, err_msg=str(shape))


def test_packed_equals_scalar_without_current_term_and_buffered_actions():
    """Model flag MG_MODEL_NO_CURRENT_ACCEL and a buffered action schedule read across many
    short graph-replayed calls."""
    n = 777
    types, vs = _fleet("mixed", n)
    acts = torch.tensor(I.commands(5, 40, n, [vs[t].n_thr for t in types]), device="cuda")
    steps = [7] * 20 + [3] * 7
    for flags in (0, MG_MODEL_NO_CURRENT_ACCEL):
        ref = _run(types, vs, False, SHAPES[1], flags=flags, steps=steps, actions=acts)
        for shape in SHAPES:
            got = _run(types, vs, True, shape, flags=flags, steps=steps, actions=acts)
            np.testing.assert_array_equal(got, ref, err_msg=f"{shape} flags={flags}")


@pytest.mark.parametrize("epb,spl", [(128, 50), (64, 500)])
def test_packed_randomised_fleet_500_substeps_vs_oracle(epb, spl):
    vs = vehicles()
    n = 4096
    types = np.zeros(n, dtype=np.int32)
    sim = Sim(n, types, vs)
    sim.set_launch(epb, spl, True)
    sim.set_schedule(False)
    sim.set_packed(True)
    sim.randomize(1234, 0.8, 1.2, 0.2, 0.3)
    sim.reset()
    cmds = I.commands(5678, 50, n, 6)
    sim.set_actions(torch.tensor(cmds, device="cuda"), 10)
    sim.step(500)
    assert sim.sync() == 0
    got = sim.get_state().cpu().numpy().astype(np.float64)
    sim.close()
    params = I.round_f32(O.randomize(1234, oracle_nominal(vs), types, f32(0.8), f32(1.2),
                                     f32(0.2)))
    s0 = np.stack([I.round_f32(O.reset_state(1234, f32(0.3), e, 0)) for e in range(n)])
    ref = O.rollout(params, oracle_geo(vs), types, s0, cmds.astype(np.float64), 10, 500, h=H)
    err = rel_err(got, ref)
    assert err.max() <= TOL_ROLLOUT, err.max(axis=0)
    q = got[:, I.S_Q:I.S_Q + 4]
    assert np.abs(np.linalg.norm(q, axis=1) - 1.0).max() <= 1e-6


def test_packed_nonfinite_stays_in_its_half():
    """Env 17 with a NaN coefficient shares its thread with env 49 (block of 32 threads: envs t
    and t + 32): only env 17 is flagged and env 49 still follows the oracle."""
    vs = vehicles()
    n = 64
    types = np.zeros(n, dtype=np.int32)
    params = np.broadcast_to(oracle_nominal(vs)[0], (n, I.NPARAM)).copy()
    params[17, I.P_DQ] = np.nan
    s0 = I.initial_states(1, n)
    sim = Sim(n, types, vs)
    sim.set_launch(32, 50, True)
    sim.set_schedule(False)
    sim.set_packed(True)
    sim.set_params(torch.tensor(params, dtype=torch.float32, device="cuda"))
    sim.set_state(torch.tensor(s0, dtype=torch.float32, device="cuda"))
    sim.step(20)
    assert sim.sync() == 1
    mask = sim.nonfinite_mask().cpu().numpy()
    assert mask[17] == 1 and mask.sum() == 1
    got = sim.get_state().cpu().numpy().astype(np.float64)
    sim.close()
    ok = np.arange(n) != 17
    ref = O.rollout(np.where(np.isnan(params), 0.0, params)[ok], oracle_geo(vs), types[ok],
                    s0[ok], np.zeros((1, ok.sum(), 8)), 1, 20, h=H)
    assert rel_err(got[ok], ref).max() <= TOL_ROLLOUT


def test_packed_kernel_info_and_fallbacks():
    """The packed kernels fit the register file without large spills; a fleet with off-centre
    gravity ignores the packed setting (general path) and still matches the scalar kernels."""
    vs = vehicles()
    for types in (np.zeros(300, np.int32), I.mixed_fleet(3, 300, max_group=80)):
        sim = Sim(len(types), types, vs)
        sim.set_packed(True)
        sim.set_schedule(False)
        info = sim.kernel_info()
        assert info["regs"] <= 255 and info["local_bytes"] <= 512, info
        sim.close()
    n = 300
    types = I.mixed_fleet(3, n, max_group=80)
    params = I.perturbed_params(3, oracle_nominal(vs)[types], n)
    params[:, I.P_RG:I.P_RG + 3] = I.round_f32(
        np.random.default_rng(2).uniform(-0.02, 0.02, (n, 3)))
    states = I.random_states(5, n, [vs[t].n_thr for t in types])
    out = []
    for packed in (False, True):
        sim = Sim(n, types, vs)
        sim.set_packed(packed)
        sim.set_params(torch.tensor(params, dtype=torch.float32, device="cuda"))
        sim.set_state(torch.tensor(states, dtype=torch.float32, device="cuda"))
        sim.set_procedural_actions(4, 10)
        sim.step(100)
        assert sim.sync() == 0
        out.append(sim.get_state().cpu().numpy())
        sim.close()
    np.testing.assert_array_equal(out[1], out[0])

