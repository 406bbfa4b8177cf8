"""mg_step_noalloc: the work-queue step for callers that must not allocate device memory while
they step (a control loop whose memory is fixed up front, a process whose memory pool is capped).
Its scheduler words live in a fixed device array inside the library; this checks, through the C
ABI, that it gives what mg_step gives on two calls in a row, that it leaves device memory use
unchanged once set up, and that it refuses fleets beyond the array's size."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2410_14117_gb300 import inputs as I
from paper_2410_14117_gb300._lib import MGError, call
from paper_2410_14117_gb300.sim import Sim

from _helpers import TOL_ROLLOUT, rel_err

pytestmark = pytest.mark.gpu


def _fleet(n, types, vs):
    sim = Sim(n, types, vs)
    sim.set_launch(128, 50, False)
    sim.set_schedule(True, True, 8)
    sim.randomize(31, 0.8, 1.2, 0.2, 0.3)
    sim.reset()
    sim.set_procedural_actions(17, 10)
    return sim


def test_noalloc_step_matches_mg_step_on_two_calls():
    """Same work-queue kernel, same schedule: the two entry points agree bit for bit."""
    vs = I.fleet_vehicles()
    n = 20000
    types = I.mixed_fleet(5, n, max_group=3000)
    ref, nal = _fleet(n, types, vs), _fleet(n, types, vs)
    for _ in range(2):
        ref.step(300)
        call("mg_step_noalloc", nal._h, 300)
        a = ref.get_state()
        b = nal.get_state()
        assert torch.isfinite(b).all()
        assert torch.equal(b, a)
    assert nal.sync() == 0
    ref.close()
    nal.close()


def test_noalloc_step_matches_static_grid_mg_step():
    """A sim whose own schedule is the static grid still gets the work-queue kernel from
    mg_step_noalloc; the two schedules round the same arithmetic alike, so the results agree
    within the rollout tolerance (and in practice exactly)."""
    vs = I.fleet_vehicles()
    n = 5000
    types = I.mixed_fleet(6, n, max_group=1500)
    ref, nal = _fleet(n, types, vs), _fleet(n, types, vs)
    ref.set_schedule(False, False)
    ref.set_launch(64, 100, True)
    for _ in range(2):
        ref.step(250)
        call("mg_step_noalloc", nal._h, 250)
        a = ref.get_state().double().cpu().numpy()
        b = nal.get_state().double().cpu().numpy()
        assert np.isfinite(b).all()
        assert rel_err(b, a).max() <= TOL_ROLLOUT
    assert nal.sync() == 0 and ref.sync() == 0
    ref.close()
    nal.close()


def test_noalloc_step_allocates_nothing_after_setup():
    vs = I.fleet_vehicles()
    n = 4096
    sim = _fleet(n, np.zeros(n, dtype=np.int32), vs)
    call("mg_step_noalloc", sim._h, 50)  # first call on the device: address look-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        call("mg_step_noalloc", sim._h, 100)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    sim.close()


def test_noalloc_rejects_fleets_beyond_the_array():
    vs = I.fleet_vehicles()
    n = 65536 * 32 + 32
    sim = Sim(n, np.zeros(n, dtype=np.int32), vs)
    with pytest.raises(MGError) as ei:
        call("mg_step_noalloc", sim._h, 1)
    assert ei.value.code == "MG_EINVAL" and "65536" in str(ei.value)
    sim.close()
