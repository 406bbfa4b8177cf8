"""Serving: continuous batching over the native job pool.  A job's result is the same alone and
in a mix (bit for bit: same kernel, draws keyed by the job's own seeds and local env ids), equals
the plain fleet API doing the same rollout, and matches the FP64 oracle; admission respects the
HBM budget and the arena's free ranges."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2410_14117_gb300 import inputs as I
from paper_2410_14117_gb300._lib import MGError
from paper_2410_14117_gb300.serve import NativeServer, Pool, Request, Server
from paper_2410_14117_gb300.sim import Sim

from _helpers import TOL_ROLLOUT, f32, oracle_geo, oracle_nominal, rel_err, vehicles

pytestmark = pytest.mark.gpu


def _requests(seed=3, n_jobs=10):
    g = np.random.default_rng(seed)
    out = []
    for i in range(n_jobs):
        out.append(Request(arrival_s=0.0005 * i, n_envs=int(g.integers(1, 3000)),
                           horizon=int(g.integers(30, 260)), vehicle=int(g.integers(0, 2)),
                           param_seed=int(g.integers(1, 2**40)),
                           cmd_seed=int(g.integers(1, 2**40)), hold=int(g.integers(1, 12))))
    return out


def _by_key(done):
    return {(r.param_seed, r.cmd_seed): r for r in done}


def test_alone_equals_mix_and_plain_fleet():
    vs = vehicles()
    reqs = _requests()
    srv = Server(vs, budget_bytes=8e9, capacity_envs=1 << 16, k=25, keep_results=True)
    mix, stats = srv.run([Request(**{k: getattr(r, k) for k in ("arrival_s", "n_envs", "horizon",
                                                              "vehicle", "param_seed",
                                                              "cmd_seed", "hold")})
                          for r in reqs], mode="batched")
    srv.close()
    assert stats["jobs"] == len(reqs)
    srv = Server(vs, budget_bytes=8e9, capacity_envs=1 << 16, k=25, keep_results=True)
    alone, _ = srv.run(reqs, mode="serial")
    srv.close()
    a, m = _by_key(alone), _by_key(mix)
    for key, r in a.items():
        torch.testing.assert_close(m[key].final_state, r.final_state, rtol=0, atol=0)
        torch.testing.assert_close(m[key].traj, r.traj, rtol=0, atol=0)
    # the plain fleet API with the same seeds gives the same rollout
    for r in list(a.values())[:4]:
        sim = Sim(r.n_envs, np.full(r.n_envs, r.vehicle), vs)
        sim.randomize(r.param_seed, 0.8, 1.2, 0.2, 0.3)
        sim.reset()
        sim.set_procedural_actions(r.cmd_seed, r.hold)
        sim.step(r.horizon)
        torch.testing.assert_close(sim.get_state()[:, :13], r.final_state[:, :13], rtol=1e-5,
                                   atol=1e-5)
        sim.close()


def test_tick_register_budget_does_not_change_results():
    """Ticks of at most 2 x SMs blocks run the 200-register kernel, larger ones the 128-register
    kernel: a 45,000-env job (352 blocks) served with three small jobs, then each job alone,
    gives the same final states and trajectories bit for bit, whichever budget its ticks got."""
    vs = vehicles()
    reqs = [Request(arrival_s=0.0, n_envs=45000, horizon=120, vehicle=0, param_seed=5,
                    cmd_seed=6, hold=10)]
    g = np.random.default_rng(11)
    for i in range(3):
        reqs.append(Request(arrival_s=0.0, n_envs=int(g.integers(100, 2000)), horizon=180,
                            vehicle=i % 2, param_seed=int(g.integers(1, 2**40)),
                            cmd_seed=int(g.integers(1, 2**40)), hold=7))
    keys = ("arrival_s", "n_envs", "horizon", "vehicle", "param_seed", "cmd_seed", "hold")
    srv = Server(vs, budget_bytes=8e9, capacity_envs=1 << 16, k=25, keep_results=True)
    mix, stats = srv.run([Request(**{k: getattr(r, k) for k in keys}) for r in reqs],
                         mode="batched")
    srv.close()
    assert stats["jobs"] == len(reqs)
    srv = Server(vs, budget_bytes=8e9, capacity_envs=1 << 16, k=25, keep_results=True)
    alone, _ = srv.run(reqs, mode="serial")
    srv.close()
    a, m = _by_key(alone), _by_key(mix)
    for key, r in a.items():
        torch.testing.assert_close(m[key].final_state, r.final_state, rtol=0, atol=0)
        torch.testing.assert_close(m[key].traj, r.traj, rtol=0, atol=0)


def test_served_job_matches_oracle():
    vs = vehicles()
    r = Request(arrival_s=0.0, n_envs=700, horizon=300, vehicle=1, param_seed=77, cmd_seed=88,
                hold=10)
    srv = Server(vs, budget_bytes=4e9, capacity_envs=1 << 14, k=50, keep_results=True)
    (res,), _ = srv.run([r], mode="batched")
    srv.close()
    types = np.full(r.n_envs, 1, dtype=np.int32)
    params = I.round_f32(O.randomize(77, oracle_nominal(vs), types, f32(0.8), f32(1.2),
                                     f32(0.2)))
    s0 = np.stack([I.round_f32(O.reset_state(77, f32(0.3), e, 0)) for e in range(r.n_envs)])
    cmds = np.stack([np.stack([O.commands(88, e, sg, 8) for e in range(r.n_envs)])
                     for sg in range(30)])
    ref, traj = O.rollout(params, oracle_geo(vs), types, s0, cmds, 10, 300, record=True)
    got = res.final_state.double().cpu().numpy()
    assert rel_err(got, ref).max() <= TOL_ROLLOUT
    g = res.traj.double().cpu().numpy()  # [T, 13, n]
    np.testing.assert_allclose(g[150].T, traj[150, :, :13], rtol=0, atol=1e-4)


def test_budget_and_capacity_bound_admission():
    vs = vehicles()
    reqs = _requests(seed=5, n_jobs=12)
    # a small arena forces jobs to wait for free ranges; a small budget forces waits too
    per = max(r.horizon * 13 * 4 * r.n_envs for r in reqs)
    srv = Server(vs, budget_bytes=4096 * 500 + 2.5 * per, capacity_envs=4096, k=40)
    base = srv.used
    done, stats = srv.run(reqs, mode="batched")
    assert stats["jobs"] == len(reqs)
    assert base < srv.peak_used <= srv.budget
    assert srv.used == base
    info = srv.pool.info()
    assert info["free_envs"] == 4096 and info["largest_free_range"] == 4096
    srv.close()


def test_pool_ranges_coalesce_and_reject():
    vs = vehicles()
    pool = Pool(1000, vs)
    a = pool.admit(300, 0, 10, 1, 2)
    b = pool.admit(300, 1, 10, 3, 4)
    c = pool.admit(300, 0, 10, 5, 6)
    assert pool.admit(200, 0, 10, 7, 8) is None          # only 100 left
    pool.release(b)
    assert pool.info()["largest_free_range"] == 300
    pool.release(a)
    assert pool.info()["largest_free_range"] == 600       # merged with the freed neighbour
    d = pool.admit(550, 1, 10, 9, 10)
    assert d is not None
    pool.tick(10)
    pool.sync()
    assert pool.progress(d) == (10, 10) and pool.progress(c) == (10, 10)
    pool.close()


def _copy(reqs):
    keys = ("arrival_s", "n_envs", "horizon", "vehicle", "param_seed", "cmd_seed", "hold")
    return [Request(**{k: getattr(r, k) for k in keys}) for r in reqs]


def test_native_server_alone_equals_mix_and_python_loop():
    """The native request loop (mg_server_*): every job's final state and trajectory record is
    the same in the mix, served one at a time, and through the Python loop, bit for bit."""
    vs = vehicles()
    reqs = _requests(seed=7, n_jobs=12)
    out = {}
    for name, cls, mode in [("mix", NativeServer, "batched"), ("alone", NativeServer, "serial"),
                            ("python", Server, "batched")]:
        srv = cls(vs, budget_bytes=8e9, capacity_envs=1 << 16, k=25, keep_results=True)
        done, stats = srv.run(_copy(reqs), mode=mode)
        srv.close()
        assert stats["jobs"] == len(reqs)
        assert all(r.admitted_s >= r.arrival_s - 1e-9 and r.done_s >= r.admitted_s for r in done)
        out[name] = _by_key(done)
    for key, r in out["alone"].items():
        for other in ("mix", "python"):
            torch.testing.assert_close(out[other][key].final_state, r.final_state, rtol=0, atol=0)
            torch.testing.assert_close(out[other][key].traj, r.traj, rtol=0, atol=0)


def test_native_server_budget_capacity_and_rejections():
    vs = vehicles()
    reqs = _requests(seed=5, n_jobs=12)
    per = max(r.horizon * 13 * 4 * r.n_envs for r in reqs)
    srv = NativeServer(vs, budget_bytes=4096 * 500 + 2.5 * per, capacity_envs=4096, k=40)
    done, stats = srv.run(_copy(reqs), mode="batched")
    assert stats["jobs"] == len(reqs)
    assert srv.arena_bytes < srv.peak_used <= srv.budget
    info = srv.pool.info()
    assert info["free_envs"] == 4096 and info["largest_free_range"] == 4096 and info["jobs"] == 0
    # FIFO: admission order follows arrival order
    order = sorted(done, key=lambda r: r.admitted_s)
    assert [r.arrival_s for r in order] == sorted(r.arrival_s for r in order)
    with pytest.raises(ValueError):
        srv.run([Request(0.0, 5000, 10, 0, 1, 2)])  # larger than the arena
    srv.close()
    # the ABI itself rejects what can never run
    from paper_2410_14117_gb300._lib import ServerConfig, JobSpec, Ranges, call
    import ctypes
    pool = Pool(1000, vs)
    h = ctypes.c_void_p()
    with pytest.raises(MGError):
        call("mg_server_create", pool._h, ctypes.byref(ServerConfig(1e9, 0, 2, 1, 0, 0, 0, 1.0)),
             ctypes.byref(h))
    call("mg_server_create", pool._h, ctypes.byref(ServerConfig(1e6, 10, 2, 1, 0, 0, 0, 1.0)),
         ctypes.byref(h))
    tk = ctypes.c_int64()
    for spec in (JobSpec(2000, 0, 10, 10, 0, 1, 2, Ranges(0.8, 1.2, 0.2, 0.3, 0)),   # > arena
                 JobSpec(100, 0, 10, 1000, 0, 1, 2, Ranges(0.8, 1.2, 0.2, 0.3, 0))):  # > budget
        with pytest.raises(MGError) as ei:
            call("mg_server_submit", h, ctypes.byref(spec), ctypes.byref(tk))
        assert ei.value.code == "MG_EINVAL"
    with pytest.raises(MGError) as ei:
        call("mg_server_job_result", h, 0, None, None)
    assert ei.value.code == "MG_EINVAL"
    call("mg_server_destroy", h)
    pool.close()



def test_native_server_wait_times_out_and_stays_usable():
    """A poll whose wait for a tick outlasts wait_timeout_s returns MG_ETIMEOUT and leaves the
    server consistent: later polls pick the job up once the device has finished it, with the
    result of an unhurried server (no fault is provoked: the tick simply takes longer than the
    1-microsecond limit)."""
    import ctypes
    from paper_2410_14117_gb300._lib import JobSpec, Ranges, ServerConfig, call
    vs = vehicles()
    pool = Pool(1 << 16, vs)
    spec = JobSpec(1 << 16, 0, 10, 600, 0, 11, 12, Ranges(0.8, 1.2, 0.2, 0.3, 0))
    results = []
    for timeout in (30.0, 1e-6):
        h = ctypes.c_void_p()
        call("mg_server_create", pool._h,
             ctypes.byref(ServerConfig(1e10, 600, 1, 1, 0, 1, 0, timeout)), ctypes.byref(h))
        tk = ctypes.c_int64()
        call("mg_server_submit", h, ctypes.byref(spec), ctypes.byref(tk))
        counts = [ctypes.c_int32() for _ in range(3)]
        timeouts = 0
        for _ in range(100000):
            try:
                call("mg_server_poll", h, *[ctypes.byref(c) for c in counts])
            except MGError as e:
                assert e.code == "MG_ETIMEOUT"
                timeouts += 1
                continue
            if not any(c.value for c in counts):
                break
        done = ctypes.c_double()
        call("mg_server_job", h, tk, None, None, ctypes.byref(done))
        assert done.value > 0.0
        state = torch.empty((1 << 16, 21), device="cuda")
        call("mg_server_job_result", h, tk, _ptr_of(state), None)
        call("mg_server_release", h, tk)
        call("mg_server_destroy", h)
        results.append((timeouts, state))
    assert results[0][0] == 0 and results[1][0] > 0
    torch.testing.assert_close(results[1][1], results[0][1], rtol=0, atol=0)
    pool.close()


def _ptr_of(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())


def _serve_jobs(pool, jobs, k=50):
    """Admit jobs (kwargs of Pool.admit plus n_envs / horizon), tick to completion, return
    (final state, trajectory) per job."""
    ids = []
    for j in jobs:
        traj = torch.empty((j["horizon"], 13, j["n_envs"]), device="cuda")
        ids.append((pool.admit(traj=traj, **j), traj))
    while pool.tick(k):
        pass
    pool.sync()
    out = [(pool.job_state(i, j["n_envs"]), t) for (i, t), j in zip(ids, jobs)]
    for i, _ in ids:
        pool.release(i)
    return out


def test_offdiag_job_alone_equals_mix_and_matches_oracle():
    """A job admitted with the off-diagonal extension (full M_A and D_l, randomised r_g) runs on
    the general path in its own launch of each tick: served alone (extension from host memory)
    or between two plain jobs (from device memory) it gives the same final state and trajectory
    bit for bit, the plain jobs give what they give without it, and it matches the FP64 oracle."""
    vs = vehicles()
    n, T, rg = 600, 200, f32(0.02)
    types = np.zeros(n, dtype=np.int32)
    params = I.round_f32(O.randomize(91, oracle_nominal(vs), types, f32(0.8), f32(1.2),
                                     f32(0.2), rg_halfwidth=rg))
    xpar = I.hydro_offdiag(93, params)
    xjob = dict(n_envs=n, vehicle_type=0, horizon=T, param_seed=91, cmd_seed=92, hold=10,
                rg_halfwidth=rg)
    plain = [dict(n_envs=1000, vehicle_type=1, horizon=150, param_seed=5, cmd_seed=6, hold=7),
             dict(n_envs=300, vehicle_type=0, horizon=250, param_seed=8, cmd_seed=9, hold=3)]
    pool = Pool(1 << 13, vs)
    (alone,) = _serve_jobs(pool, [dict(xjob, xh=xpar.astype(np.float32))])
    ref_plain = _serve_jobs(pool, plain)
    mix = _serve_jobs(pool, [plain[0], dict(xjob, xh=torch.tensor(xpar, dtype=torch.float32,
                                                                   device="cuda")), plain[1]])
    pool.close()
    assert torch.equal(mix[1][0], alone[0]) and torch.equal(mix[1][1], alone[1])
    for (fs, tr), (rfs, rtr) in zip([mix[0], mix[2]], ref_plain):
        assert torch.equal(fs, rfs) and torch.equal(tr, rtr)
    s0 = np.stack([I.round_f32(O.reset_state(91, f32(0.3), e, 0)) for e in range(n)])
    cmds = np.stack([np.stack([O.commands(92, e, sg, 6) for e in range(n)])
                     for sg in range(T // 10)])
    ref, traj = O.rollout(params, oracle_geo(vs), types, s0, cmds, 10, T, record=True, xpar=xpar)
    got = alone[0].double().cpu().numpy()
    assert rel_err(got, ref).max() <= TOL_ROLLOUT
    g = alone[1].double().cpu().numpy()
    np.testing.assert_allclose(g[100].T, traj[100, :, :13], rtol=0, atol=1e-4)
    # the extension changes the rollout (it is not silently dropped)
    ref0 = O.rollout(params, oracle_geo(vs), types, s0, cmds, 10, T)
    assert rel_err(got, ref0).max() > 100 * TOL_ROLLOUT


def test_offdiag_admission_checks():
    vs = vehicles()
    pool = Pool(1000, vs)
    with pytest.raises(ValueError):
        pool.admit(100, 0, 10, 1, 2, xh=np.zeros((100, 44), np.float32))
    with pytest.raises(MGError) as ei:   # r_g randomisation needs the extension or an r_g pool
        pool.admit(100, 0, 10, 1, 2, rg_halfwidth=0.01)
    assert ei.value.code == "MG_EINVAL"
    a = pool.admit(100, 0, 10, 1, 2, rg_halfwidth=0.01, xh=np.zeros((100, 45), np.float32))
    assert a is not None
    pool.release(a)
    pool.close()


def test_native_server_serves_offdiag_jobs():
    """Jobs with the off-diagonal extension through the native request loop
    (mg_server_submit_offdiag, records from host and from device memory): each job's final
    state and trajectory are the same in the mix, one at a time and through the Python loop, bit
    for bit, and the extension is applied (the same job without it ends elsewhere)."""
    vs = vehicles()
    reqs = _requests(seed=9, n_jobs=8)
    for i in (1, 4, 6):
        r = reqs[i]
        nominal = np.repeat(oracle_nominal(vs)[r.vehicle][None], r.n_envs, axis=0)
        x = I.hydro_offdiag(300 + i, nominal, 0.1).astype(np.float32)
        r.xh = x if i != 4 else torch.tensor(x, device="cuda")
    keys = ("arrival_s", "n_envs", "horizon", "vehicle", "param_seed", "cmd_seed", "hold", "xh")
    out = {}
    for name, cls, mode in [("mix", NativeServer, "batched"), ("alone", NativeServer, "serial"),
                            ("python", Server, "batched")]:
        srv = cls(vs, budget_bytes=8e9, capacity_envs=1 << 16, k=25, keep_results=True)
        done, stats = srv.run([Request(**{k: getattr(r, k) for k in keys}) for r in reqs],
                              mode=mode)
        srv.close()
        assert stats["jobs"] == len(reqs)
        out[name] = _by_key(done)
    for key, r in out["alone"].items():
        for other in ("mix", "python"):
            torch.testing.assert_close(out[other][key].final_state, r.final_state, rtol=0, atol=0)
            torch.testing.assert_close(out[other][key].traj, r.traj, rtol=0, atol=0)
    plain = reqs[1]
    srv = NativeServer(vs, budget_bytes=8e9, capacity_envs=1 << 16, k=25, keep_results=True)
    (res,), _ = srv.run([Request(**{k: getattr(plain, k) for k in keys[:-1]})], mode="batched")
    srv.close()
    key = (plain.param_seed, plain.cmd_seed)
    assert (res.final_state - out["mix"][key].final_state).abs().max() > 1e-3
