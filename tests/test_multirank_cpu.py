"""The multi-rank path on CPU (world size 2, gloo): every rank integrates its own fleet with env
ids offset by rank, as bench.py does under torchrun (no collective in the data path), and the
slowest rank's time is the job's.  The union of the shards must equal the single-process fleet,
which holds because every draw is keyed by the global env id.  The one collective of the
sharded adjoint (the gradient of coefficients shared by the whole fleet) is checked the same
way."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shard(gid0, n, steps):
    from oracle import oracle as O
    from paper_2410_14117_gb300 import inputs as I
    vs = I.fleet_vehicles()
    nominal = np.stack([I.round_f32(v.params) for v in vs])
    geo = np.stack([I.round_f32(v.geo()) for v in vs])
    types = np.zeros(n, dtype=np.int32)
    par = I.round_f32(O.randomize(1234, nominal, types, 0.8, 1.2, 0.2, gid0=gid0))
    s0 = np.stack([I.round_f32(O.reset_state(1234, 0.3, gid0 + e, 0)) for e in range(n)])
    cmd = np.stack([np.stack([O.commands(5678, gid0 + e, sg, 6) for e in range(n)])
                    for sg in range(steps // 10)])
    return O.rollout(par, geo, types, s0, cmd, 10, steps, nthreads=1)


def _worker(rank, world, port, n, steps, out_path):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = _shard(bench.rank_env_offset(rank, n), n, steps)
    parts = [torch.zeros((n, 21), dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, torch.from_numpy(mine))
    slowest = bench.reduce_max(float(rank + 1))
    if rank == 0:
        np.save(out_path, torch.cat(parts).numpy())
        np.save(out_path + ".max.npy", np.array([slowest]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_equal_one_fleet(tmp_path):
    n, steps, world = 24, 30, 2
    out = str(tmp_path / "union.npy")
    mp.spawn(_worker, args=(world, _free_port(), n, steps, out), nprocs=world, join=True)
    union = np.load(out)
    whole = _shard(0, world * n, steps)
    np.testing.assert_array_equal(union, whole)
    assert np.load(out + ".max.npy")[0] == world


def _fake_dcoef(gid0, n):
    """Per-env coefficient gradients keyed by the global env id (stand-ins for the adjoint's
    output; the reduction does not look at their values)."""
    g = np.stack([np.random.default_rng(1000 + gid0 + e).normal(size=18) for e in range(n)])
    return g.astype(np.float32)


def _grad_worker(rank, world, port, n, out_path):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2410_14117_gb300.adjoint import shared_coefficient_grad
    mine = torch.from_numpy(_fake_dcoef(bench.rank_env_offset(rank, n), n))
    total = shared_coefficient_grad(mine)
    np.save(out_path + f".{rank}.npy", total.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_shared_coefficient_gradient_all_reduce(tmp_path):
    n, world = 16, 2
    out = str(tmp_path / "grad")
    mp.spawn(_grad_worker, args=(world, _free_port(), n, out), nprocs=world, join=True)
    whole = _fake_dcoef(0, world * n).astype(np.float64).sum(axis=0)
    for r in range(world):
        got = np.load(out + f".{r}.npy")
        np.testing.assert_allclose(got, whole, rtol=1e-5, atol=1e-5)
