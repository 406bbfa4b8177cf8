"""The serving loop's host logic on CPU, with a fake pool and fake events (no GPU): FIFO
admission under the memory budget, every job completing, a tick that never completes turning into
a TimeoutError instead of a hang, and requests that can never fit being refused up front."""
import pytest

from paper_2410_14117_gb300.serve import ARENA_BYTES_PER_ENV, Request, Server


class FakePool:
    """Stands in for the device pool: jobs advance by k sub-steps per tick."""

    def __init__(self, capacity):
        self.capacity = capacity
        self.device = "cpu"
        self.stream = None
        self.jobs = {}
        self.free = capacity
        self.admitted = []
        self.max_live = 0

    def admit(self, n_envs, vehicle, horizon, param_seed, cmd_seed, hold=10, traj=None, xh=None):
        if n_envs > self.free:
            return None
        jid = len(self.admitted)
        self.admitted.append(param_seed)
        self.jobs[jid] = [0, horizon, n_envs]
        self.free -= n_envs
        self.max_live = max(self.max_live, len(self.jobs))
        return jid

    def tick(self, k):
        live = 0
        for j in self.jobs.values():
            if j[0] < j[1]:
                j[0] = min(j[1], j[0] + k)
                live += 1
        return live

    def progress(self, jid):
        d, h, _ = self.jobs[jid]
        return d, h

    def release(self, jid):
        self.free += self.jobs.pop(jid)[2]

    def close(self):
        pass


class Event:
    def __init__(self, done=True):
        self.done = done

    def record(self, stream):
        pass

    def query(self):
        return self.done


def _requests(n=12):
    return [Request(arrival_s=0.0, n_envs=100 + 10 * i, horizon=50 + 25 * (i % 4), vehicle=0,
                    param_seed=i, cmd_seed=1000 + i, hold=10) for i in range(n)]


def test_all_jobs_complete_in_fifo_order():
    pool = FakePool(4096)
    srv = Server([], budget_bytes=1e12, k=25, pool=pool, event=Event)
    done, stats = srv.run(_requests(), mode="batched", realtime=False)
    assert stats["jobs"] == 12 and len(done) == 12
    assert pool.admitted == list(range(12))            # FIFO
    assert all(r.done_s >= r.admitted_s >= r.arrival_s for r in done)
    assert not pool.jobs and pool.free == 4096          # every job released
    assert srv.used == 4096 * ARENA_BYTES_PER_ENV < srv.peak_used  # records freed, arena kept


def test_budget_and_serial_mode_bound_residency():
    reqs = _requests(8)
    per_job = max(r.horizon * 13 * 4 * r.n_envs for r in reqs)
    pool = FakePool(4096)
    srv = Server([], budget_bytes=1e12, k=25, pool=pool, event=Event)
    arena = srv.used
    srv.budget = arena + 1.5 * per_job   # room for one or two trajectory records at a time
    srv.run(reqs, mode="batched", realtime=False)
    assert arena < srv.peak_used <= srv.budget and srv.used == arena
    assert 1 < pool.max_live < len(reqs)               # the budget, not the arena, bound it
    pool2 = FakePool(4096)
    srv2 = Server([], budget_bytes=1e12, k=25, pool=pool2, event=Event)
    srv2.run(_requests(8), mode="serial", realtime=False)
    assert pool2.max_live == 1


def test_stuck_tick_raises_timeout_instead_of_hanging():
    pool = FakePool(4096)
    srv = Server([], budget_bytes=1e12, k=25, pool=pool, event=lambda: Event(done=False),
                 wait_timeout_s=0.05)
    with pytest.raises(TimeoutError):
        srv.run(_requests(3), mode="batched", realtime=False)


def test_request_that_can_never_fit_is_refused():
    pool = FakePool(64)
    srv = Server([], budget_bytes=1e12, k=25, pool=pool, event=Event)
    with pytest.raises(ValueError):
        srv.run([Request(arrival_s=0.0, n_envs=65, horizon=10, vehicle=0, param_seed=1,
                         cmd_seed=2, hold=10)], realtime=False)
