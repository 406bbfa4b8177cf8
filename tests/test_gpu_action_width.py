"""Unpadded action schedules (mg_set_action_width 6): for a fleet of 6-thruster vehicles the
throttle schedule can be laid out [n_seg][n][6] instead of [n_seg][n][8]; every step kernel, the
asynchronous host copy and the adjoint must then give what the padded layout gives, bit for bit
(the commands are the same numbers, only their addresses change)."""
import numpy as np
import pytest
import torch

from paper_2410_14117_gb300 import inputs as I
from paper_2410_14117_gb300.adjoint import COEF_SLICE, rollout
from paper_2410_14117_gb300.sim import MGError, Sim

from _helpers import vehicles

pytestmark = pytest.mark.gpu

HOLD, K = 10, 230


def _fleet(vs, n, launch):
    sim = Sim(n, np.zeros(n, np.int32), vs)
    kind, epb, spl = launch
    sim.set_launch(epb, spl, True)
    sim.set_schedule(kind == "queue", kind != "narrow", 8 if kind == "queue" else 0)
    sim.randomize(5, 0.8, 1.2, 0.2, 0.3)
    sim.reset()
    return sim


@pytest.mark.parametrize("launch", [("static", 128, 50), ("narrow", 32, 1), ("queue", 128, 40),
                                    ("narrow", 64, 100)])
@pytest.mark.parametrize("how", ["copied", "borrowed", "async"])
def test_six_wide_schedule_equals_padded_schedule(launch, how):
    vs = vehicles()
    n = 1000 if launch[2] > 1 else 300
    pad = I.commands(77, K // HOLD + 1, n, 6)
    six = np.ascontiguousarray(pad[:, :, :6])
    ref = _fleet(vs, n, launch)
    ref.set_actions(torch.tensor(pad, device="cuda"), HOLD)
    ref.step(K)
    want = ref.get_state()
    ref.close()

    sim = _fleet(vs, n, launch)
    sim.set_action_width(6)
    if how == "copied":
        sim.set_actions(torch.tensor(six, device="cuda"), HOLD)
    elif how == "borrowed":
        six_dev = torch.tensor(six, device="cuda")
        sim.set_actions_borrowed(six_dev, HOLD)
    else:
        sim.set_actions_async(torch.from_numpy(six).pin_memory(), HOLD)
    sim.step(K - 30)
    sim.step(30)
    assert sim.sync() == 0
    assert torch.equal(sim.get_state(), want)
    sim.close()


def test_six_wide_adjoint_equals_padded_adjoint():
    vs = vehicles()
    n, T, C = 256, 60, 20
    pad = torch.tensor(I.commands(3, T // HOLD, n, 6), device="cuda")
    s0 = torch.tensor(I.initial_states(4, n), dtype=torch.float32, device="cuda")
    grads = []
    for width in (8, 6):
        sim = Sim(n, np.zeros(n, np.int32), vs)
        sim.randomize(6, 0.8, 1.2, 0.2, 0.3)
        if width == 6:
            sim.set_action_width(6)
        coeffs = sim.get_params()[:, COEF_SLICE].clone().requires_grad_(True)
        acts = (pad if width == 8 else pad[:, :, :6].contiguous()).clone().requires_grad_(True)
        traj = rollout(sim, coeffs, acts, s0, HOLD, T, C)
        loss = (traj ** 2).mean()
        gc, ga = torch.autograd.grad(loss, (coeffs, acts))
        grads.append((traj.detach(), gc, ga))
        sim.close()
    assert torch.equal(grads[0][0], grads[1][0])
    assert torch.equal(grads[0][1], grads[1][1])
    assert torch.equal(grads[0][2][:, :, :6], grads[1][2])
    assert not grads[0][2][:, :, 6:].any()


def test_width_change_clears_the_schedule_and_bad_widths_are_rejected():
    vs = vehicles()
    n = 200
    sim = _fleet(vs, n, ("static", 128, 50))
    zero = _fleet(vs, n, ("static", 128, 50))
    zero.set_actions(None, 1)
    sim.set_actions(torch.tensor(I.commands(1, 5, n, 6), device="cuda"), HOLD)
    sim.set_action_width(6)  # the padded schedule no longer applies: commands are zero
    sim.step(40)
    zero.step(40)
    assert torch.equal(sim.get_state(), zero.get_state())
    with pytest.raises(ValueError):
        sim.set_actions(torch.zeros((2, n, 8), device="cuda"), HOLD)
    for bad in (5, 7, 0):
        with pytest.raises(MGError) as ei:
            sim.set_action_width(bad)
        assert ei.value.code == "MG_EINVAL"
    sim.close()
    zero.close()
    types = I.mixed_fleet(2, 500, max_group=100)
    assert (types == 1).any() and (types == 0).any()
    mixed = Sim(500, types, vs)
    with pytest.raises(MGError) as ei:
        mixed.set_action_width(6)
    assert ei.value.code == "MG_EINVAL"
    mixed.close()
