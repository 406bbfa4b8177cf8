"""Background randomisation (mg_randomize_prefetch): a prefetched draw installed by the matching
mg_randomize gives the parameters of a direct draw bit for bit; a draw whose key does not match
(seed, ranges, env-id offset) is made directly; an episode pipeline that draws each next
episode's parameters while the current episode steps ends every episode in the states of the
plain loop, bit for bit; fleets whose mass matrices may be full are rejected."""
import copy

import numpy as np
import pytest
import torch

from paper_2410_14117_gb300 import inputs as I
from paper_2410_14117_gb300._lib import MG_NXPARAM
from paper_2410_14117_gb300.sim import MGError, Sim

from _helpers import vehicles

pytestmark = pytest.mark.gpu

K = 200
HOLD = 10


def _direct_params(types, vs, seed, lo=0.8, hi=1.2, cs=0.2, offset=0):
    sim = Sim(len(types), types, vs)
    sim.set_env_id_offset(offset)
    sim.randomize(seed, lo, hi, cs, 0.3)
    p = sim.get_params().cpu()
    sim.close()
    return p


def test_installed_prefetch_equals_direct_draw():
    vs = vehicles()
    n = 5000
    types = I.mixed_fleet(5, n, max_group=900)
    sim = Sim(n, types, vs)
    sim.randomize_prefetch(77, 0.7, 1.3, 0.25)
    sim.randomize(77, 0.7, 1.3, 0.25, 0.3)
    assert sim.sync() == 0
    torch.testing.assert_close(sim.get_params().cpu(), _direct_params(types, vs, 77, 0.7, 1.3, 0.25),
                               rtol=0, atol=0)
    # the same key again installs again; the asynchronous form installs as well
    sim.randomize(5, 0.8, 1.2, 0.2, 0.3)
    sim.randomize(77, 0.7, 1.3, 0.25, 0.3, wait=False)
    assert sim.sync() == 0
    torch.testing.assert_close(sim.get_params().cpu(), _direct_params(types, vs, 77, 0.7, 1.3, 0.25),
                               rtol=0, atol=0)
    sim.close()


@pytest.mark.parametrize("change", ["seed", "lo", "hi", "current", "offset"])
def test_mismatched_key_draws_directly(change):
    vs = vehicles()
    n = 1200
    types = np.zeros(n, dtype=np.int32)
    sim = Sim(n, types, vs)
    sim.randomize_prefetch(11, 0.8, 1.2, 0.2)
    seed, lo, hi, cs, off = 11, 0.8, 1.2, 0.2, 0
    if change == "seed":
        seed = 12
    elif change == "lo":
        lo = 0.85
    elif change == "hi":
        hi = 1.15
    elif change == "current":
        cs = 0.1
    else:
        off = 4096
        sim.set_env_id_offset(off)
    sim.randomize(seed, lo, hi, cs, 0.3)
    assert sim.sync() == 0
    got = sim.get_params().cpu()
    sim.close()
    torch.testing.assert_close(got, _direct_params(types, vs, seed, lo, hi, cs, off), rtol=0, atol=0)
    assert not torch.equal(got, _direct_params(types, vs, 11))


@pytest.mark.parametrize("queue", [False, True])
def test_pipelined_prefetch_episodes_equal_plain_loop(queue):
    vs = vehicles()
    n = 20000
    types = np.zeros(n, dtype=np.int32)
    acts = torch.tensor(I.commands(3, K // HOLD, n, 6), device="cuda")

    def run(prefetch):
        sim = Sim(n, types, vs)
        sim.set_launch(128, 100, True)
        sim.set_schedule(queue, True, 8)
        sim.set_actions_borrowed(acts, HOLD)
        outs = []
        if prefetch:
            sim.randomize_prefetch(500)
        for ep in range(5):
            sim.randomize(500 + ep, 0.8, 1.2, 0.2, 0.3, wait=False)
            sim.reset()
            sim.set_actions_borrowed(acts, HOLD)
            sim.step(K)
            if prefetch:  # the next episode's draw runs beside this episode's steps
                sim.randomize_prefetch(500 + ep + 1)
            outs.append(sim.get_state().cpu())
        assert sim.sync() == 0
        sim.close()
        return outs

    plain, piped = run(False), run(True)
    for ep, (a, b) in enumerate(zip(plain, piped)):
        torch.testing.assert_close(b, a, rtol=0, atol=0, msg=f"episode {ep}")


def test_prefetch_rejects_fleets_with_full_mass_matrices():
    vs = vehicles()
    off = copy.deepcopy(vs[0])
    off.params[I.P_RG] = 0.02
    sim = Sim(64, np.zeros(64, dtype=np.int32), [off])
    with pytest.raises(MGError) as ei:
        sim.randomize_prefetch(1)
    assert ei.value.code == "MG_EINVAL"
    sim.close()
    sim = Sim(64, np.zeros(64, dtype=np.int32), vs)
    with pytest.raises(MGError) as ei:
        sim.randomize_prefetch(1, 1.2, 0.8)
    assert ei.value.code == "MG_EINVAL"
    sim.close()
    # with the off-diagonal extension set, a draw prefetched before it is not installed (its
    # derived planes hold diagonal mass inverses): the steps equal those after a direct draw
    x = torch.zeros((64, MG_NXPARAM), device="cuda")
    x[:, 0] = 0.5
    acts = torch.tensor(I.commands(4, 5, 64, 6), device="cuda")
    outs = []
    for prefetch in (False, True):
        sim = Sim(64, np.zeros(64, dtype=np.int32), vs)
        if prefetch:
            sim.randomize_prefetch(1)
        sim.set_hydro_offdiag(x)
        if prefetch:
            with pytest.raises(MGError) as ei:
                sim.randomize_prefetch(2)
            assert ei.value.code == "MG_EINVAL"
        sim.randomize(1, 0.8, 1.2, 0.2, 0.3)
        sim.reset()
        sim.set_actions(acts, HOLD)
        sim.step(50)
        outs.append(sim.get_state().cpu())
        assert sim.sync() == 0
        sim.close()
    torch.testing.assert_close(outs[1], outs[0], rtol=0, atol=0)
