"""Asynchronous host transfers (mg_set_actions_async / mg_get_state_async) and the graph cache
keyed by the action source: a pipelined sequence of episodes through page-locked host buffers
gives the states of the synchronous calls, bit for bit; alternating action buffers replays
cached graphs with the results of direct launches."""
import numpy as np
import pytest
import torch

from paper_2410_14117_gb300 import inputs as I
from paper_2410_14117_gb300.sim import MGError, Sim

from _helpers import vehicles

pytestmark = pytest.mark.gpu

K = 120   # sub-steps per episode
HOLD = 10


def _sim(types, vs, queue):
    sim = Sim(len(types), types, vs)
    sim.set_launch(64, 40, True)
    sim.set_schedule(queue)
    return sim


@pytest.mark.parametrize("queue", [False, True])
def test_pipelined_episodes_through_pinned_host_buffers_equal_sync(queue):
    vs = vehicles()
    n = 3000
    types = I.mixed_fleet(12, n, max_group=700)
    nt = [vs[t].n_thr for t in types]
    acts = [torch.from_numpy(I.commands(40 + ep, K // HOLD, n, nt)).pin_memory()
            for ep in range(4)]
    outs = [torch.empty((n, 21), dtype=torch.float32).pin_memory() for _ in range(4)]

    ref = []
    sim = _sim(types, vs, queue)
    for ep in range(4):
        sim.randomize(100 + ep, 0.8, 1.2, 0.2, 0.3)
        sim.reset()
        sim.set_actions(acts[ep].cuda(), HOLD)
        sim.step(K)
        ref.append(sim.get_state().cpu().numpy())
    assert sim.sync() == 0
    sim.close()

    sim = _sim(types, vs, queue)
    for ep in range(4):  # every call returns at once; the copies overlap the other episodes
        sim.set_actions_async(acts[ep], HOLD)
        sim.randomize(100 + ep, 0.8, 1.2, 0.2, 0.3, wait=False)
        sim.reset()
        sim.step(K)
        sim.get_state_async(outs[ep])
    assert sim.sync() == 0
    for ep in range(4):
        np.testing.assert_array_equal(outs[ep].numpy(), ref[ep], err_msg=f"episode {ep}")
    # switching back to the synchronous setters after asynchronous buffers
    sim.set_actions(acts[0].cuda(), HOLD)
    sim.randomize(100, 0.8, 1.2, 0.2, 0.3)
    sim.reset()
    sim.step(K)
    np.testing.assert_array_equal(sim.get_state().cpu().numpy(), ref[0])
    sim.close()


def test_async_transfers_reject_pageable_and_device_memory():
    vs = vehicles()
    n = 64
    sim = Sim(n, np.zeros(n, np.int32), vs)
    pageable = torch.zeros((3, n, 8))
    for bad in (pageable, pageable.cuda()):
        with pytest.raises(MGError) as ei:
            sim.set_actions_async(bad, 10)
        assert ei.value.code == "MG_EINVAL"
    for bad in (torch.zeros((n, 21)), torch.zeros((n, 21), device="cuda")):
        with pytest.raises(MGError) as ei:
            sim.get_state_async(bad)
        assert ei.value.code == "MG_EINVAL"
    with pytest.raises(MGError):
        sim.set_actions_async(torch.zeros((0, n, 8)).pin_memory(), 10)
    sim.close()


@pytest.mark.parametrize("queue", [False, True])
def test_alternating_action_buffers_replay_cached_graphs(queue):
    """Borrowed device buffers A, B, A, B, ... with graph replay: every switch keeps the cached
    graphs (the key includes the buffer) and the results equal direct launches."""
    vs = vehicles()
    n = 1500
    types = I.mixed_fleet(5, n, max_group=400)
    nt = [vs[t].n_thr for t in types]
    bufs = [torch.tensor(I.commands(60 + i, 6, n, nt), device="cuda") for i in range(2)]
    out = []
    for graph in (False, True):
        sim = Sim(n, types, vs)
        sim.set_launch(96, 20, graph)
        sim.set_schedule(queue)
        sim.randomize(3, 0.8, 1.2, 0.2, 0.3)
        sim.reset()
        for r in range(6):
            sim.set_actions_borrowed(bufs[r % 2], 10)
            sim.step(30)
            sim.step(30)
        sim.set_procedural_actions(7, 5)
        sim.step(30)
        sim.set_procedural_actions(8, 5)
        sim.step(30)
        assert sim.sync() == 0
        out.append(sim.get_state().cpu().numpy())
        sim.close()
    np.testing.assert_array_equal(out[1], out[0])


@pytest.mark.parametrize("n", [1, 127, 128, 129, 1000])
@pytest.mark.parametrize("offset", [0, 1, 3])
def test_state_rows_round_trip_any_alignment_and_ragged_tail(n, offset):
    """mg_set_state / mg_get_state move [n][21] rows through shared memory in 128-row spans,
    as 16-byte vectors when the buffer is 16-byte aligned: every fleet size (ragged last span)
    and buffer offset (1 or 3 floats: misaligned) gives the rows back bit for bit."""
    vs = vehicles()
    sim = Sim(n, np.zeros(n, dtype=np.int32), vs)
    rows = torch.from_numpy(I.random_states(7 + n, n, 6).astype(np.float32)).cuda()
    src = torch.full((n * 21 + offset,), float("nan"), device="cuda")
    src[offset:] = rows.reshape(-1)
    sim.set_state(src[offset:].view(n, 21))
    dst = torch.full((n * 21 + offset + 5,), -7.0, device="cuda")
    sim.get_state(dst[offset:offset + n * 21].view(n, 21))
    host = sim.get_state(torch.empty((n, 21), dtype=torch.float32))
    assert sim.sync() == 0
    sim.close()
    torch.testing.assert_close(dst[offset:offset + n * 21].view(n, 21), rows, rtol=0, atol=0)
    assert torch.all(dst[:offset] == -7.0) and torch.all(dst[offset + n * 21:] == -7.0)
    torch.testing.assert_close(host, rows.cpu(), rtol=0, atol=0)
