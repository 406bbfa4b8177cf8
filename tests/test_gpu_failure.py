"""Failure detection on the GPU without a fault: the work-queue schedule's bounded device-side
wait is made to run out (a limit of a few polls against a chunk that takes tens of
microseconds), the launch still ends, mg_sync reports MG_ETIMEOUT once, and after the limit is
restored the same sim steps to the oracle's result again."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2410_14117_gb300 import inputs as I
from paper_2410_14117_gb300.sim import MGError, Sim

from _helpers import TOL_ROLLOUT, f32, oracle_geo, oracle_nominal, rel_err, vehicles

pytestmark = pytest.mark.gpu

SEED, HOLD, K, CHUNK = 21, 10, 400, 100


def _fleet(vs, n, cmds):
    sim = Sim(n, np.zeros(n, np.int32), vs)
    sim.set_launch(128, CHUNK, False)
    sim.set_schedule(True, True, 8)
    sim.randomize(SEED, 0.8, 1.2, 0.2, 0.3)
    sim.reset()
    sim.set_actions(cmds, HOLD)
    return sim


def test_work_queue_wait_times_out_then_recovers():
    vs = vehicles()
    # 64 envs: two 32-env slices, one block of four warps.  The warps claim units 0..3 at once,
    # so two of them start on chunk 1 of a slice whose chunk 0 is still running and must wait.
    n = 64
    cmds_np = I.commands(22, K // HOLD, n, 6)
    cmds = torch.tensor(cmds_np, device="cuda")
    sim = _fleet(vs, n, cmds)
    s0 = sim.get_state().clone()

    sim.set_wait_limit(2)  # ~0.3 us against ~60 us per chunk: the waits must give up
    sim.step(K)
    with pytest.raises(MGError) as ei:
        sim.sync()
    assert ei.value.code == "MG_ETIMEOUT"
    assert "timed out" in str(ei.value)
    assert sim.sync() == 0  # reported once; the racing units still left finite states

    # restored limit, restored start state: the normal result, bit for bit and vs the oracle
    sim.set_wait_limit(0)
    sim.set_state(s0)
    sim.set_actions(cmds, HOLD)
    sim.step(K)
    assert sim.sync() == 0
    got = sim.get_state()
    ref_sim = _fleet(vs, n, cmds)
    ref_sim.step(K)
    assert ref_sim.sync() == 0
    assert torch.equal(got, ref_sim.get_state())
    sim.close()
    ref_sim.close()

    types = np.zeros(n, np.int32)
    par = I.round_f32(O.randomize(SEED, oracle_nominal(vs), types, f32(0.8), f32(1.2), f32(0.2)))
    st0 = np.stack([I.round_f32(O.reset_state(SEED, f32(0.3), e, 0)) for e in range(n)])
    ref = O.rollout(par, oracle_geo(vs), types, st0, cmds_np.astype(np.float64), HOLD, K, h=0.01)
    err = rel_err(got.double().cpu().numpy(), ref)
    assert err.max() <= TOL_ROLLOUT, err.max(axis=0)


def test_wait_limit_rejects_out_of_range():
    vs = vehicles()
    sim = Sim(32, np.zeros(32, np.int32), vs)
    with pytest.raises(MGError) as ei:
        sim.set_wait_limit(1 << 31)
    assert ei.value.code == "MG_EINVAL"
    sim.close()
