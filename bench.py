#!/usr/bin/env python
"""Benchmark: env-steps/s of the fused persistent Fossen step on domain-randomised fleets.

One benchmark step is one episode over the whole hot path: domain randomisation with the FP64
mass-matrix inverse, reset, loading the episode's throttle schedule, 1,000 RK4 sub-steps
(persistent kernel, 50 sub-steps per launch, replayed from one CUDA graph) and the state
read-back.  Prints one JSON line.

  python bench.py [--gpus N --steps K --warmup W]     # this library (default)
  python bench.py --impl reference ...                 # the FP64 CPU oracle on the host cores

Under torchrun (N > 1) every rank steps its own fleet (env ids offset by rank: weak scaling, no
collective in the data path); the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/s at 64K envs (fused vs per-step, same GPU); p50/p99 serve latency"

# Algorithmic FP32 work per env and sub-step of the diagonal-mass step (FMA = 2 flops, a product
# into a zero accumulator 1), counted from the arithmetic of Eq. 1 + RK4 as the kernel performs
# it for the vectored thruster layout (the allocation's known zeros are not multiplied): 4
# right-hand sides without the lag derivative (6 thrusters: 223 flops each = thrust 52, R(q) 28,
# relative velocity 18, translational rows 45, rotational rows 45, kinematics 35; 8 thrusters:
# 237) + RK4 stage updates and combination of p, q, nu (164; the unused stage values of p are
# not formed) + the throttle lag in its closed form (12 per thruster) + quaternion
# renormalisation (15).
FLOPS_PER_ENV_STEP = {6: 4 * 223 + 164 + 6 * 12 + 15, 8: 4 * 237 + 164 + 8 * 12 + 15}
# Algorithmic HBM bytes per env of one launch: state read + written ((13 + n_thr) floats each),
# the 34 parameter floats of the diagonal-mass step, and one command row (unpadded for a fleet of
# 6-thruster vehicles: mg_set_action_width 6).
STATE_BYTES = {6: 19 * 4, 8: 21 * 4}
PARAM_BYTES = 34 * 4
CMD_BYTES = {6: 6 * 4, 8: 8 * 4}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-envs", type=int, default=65536)
    ap.add_argument("--horizon", type=int, default=1000)
    ap.add_argument("--k", type=int, default=50, help="sub-steps per persistent launch")
    ap.add_argument("--epb", type=int, default=128, help="envs per block")
    ap.add_argument("--hold", type=int, default=10)
    ap.add_argument("--no-per-step", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (static grid)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the mixed-fleet, adjoint and serving sections")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers

def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_alu_peak_tflops(sm_mhz, n_sm=152):
    # 4 sub-partitions x 32 FP32 lanes per SM, one FMA (2 flops) per lane per cycle.
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.path = None
        self.dev = device_index

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 8:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# Sources each profiled step kernel is compiled from; a committed ncu capture describes a kernel
# only while its files are unchanged.
_COMMON_SOURCES = ("paper_2410_14117_gb300/csrc/mg_advance.cuh",
                   "paper_2410_14117_gb300/csrc/mg_device.cuh",
                   "paper_2410_14117_gb300/csrc/mg_internal.h",
                   "include/mg.h")
KERNEL_SOURCES = {
    "k_fleet": ("paper_2410_14117_gb300/csrc/mg_step.cu",) + _COMMON_SOURCES,
    "k_fleet_queue": ("paper_2410_14117_gb300/csrc/mg_step.cu",) + _COMMON_SOURCES,
    "k_fleet_step1": ("paper_2410_14117_gb300/csrc/mg_step.cu",) + _COMMON_SOURCES,
}


def kernel_sources_sha(files) -> str:
    """Hash of the code of the sources a kernel is compiled from (comments removed, whitespace
    collapsed: an edit of the documentation alone keeps the kernel), to tell whether a committed
    ncu capture still describes the kernel being timed."""
    import hashlib
    import re
    h = hashlib.sha256()
    for rel in files:
        h.update(rel.encode())
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, n_envs: int, k: int):
    """DRAM bytes (read + write) of one launch of `k` sub-steps over `n_envs` envs, from
    profiles/dram_traffic.txt: a capture of the current sources with the same sub-steps per
    launch and fleet size (whether the working set stays in the L2 depends on the size), else
    None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path) or kernel not in KERNEL_SOURCES:
        return None
    sha = kernel_sources_sha(KERNEL_SOURCES[kernel])
    for line in open(path):
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if (f.get("kernel") == kernel and f.get("sources_sha") == sha and int(f["k"]) == k
                and int(f["n_envs"]) == n_envs):
            return float(f["dram_bytes"])
    return None


def reduce_max(x: float, device="cpu") -> float:
    """Maximum of x over the ranks of the default process group (x itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_env_offset(rank: int, n_envs: int) -> int:
    """First global env id of a rank's fleet (weak scaling: every rank steps n_envs envs)."""
    return rank * n_envs


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------- CPU baseline

def cpu_baseline(n_envs, horizon, hold, target_s=12.0):
    """The FP64 oracle as it stands, on the host cores, over a bounded sample of the same
    workload (randomised BlueROV2 fleet with current, same command process): episodes of
    min(n_envs, 8192) envs x horizon sub-steps, repeated until about target_s seconds."""
    import numpy as np
    from oracle import oracle as O
    from paper_2410_14117_gb300 import inputs as I

    vs = I.fleet_vehicles()
    nominal = np.stack([I.round_f32(v.params) for v in vs])
    geo = np.stack([I.round_f32(v.geo()) for v in vs])
    ns = min(n_envs, 8192)
    types = np.zeros(ns, dtype=np.int32)
    par = I.round_f32(O.randomize(1234, nominal, types, float(np.float32(0.8)),
                                  float(np.float32(1.2)), float(np.float32(0.2))))
    s0 = I.initial_states(21, ns)
    cmd = I.commands(5678, max(1, math.ceil(horizon / hold)), ns, 6).astype(np.float64)
    t = time.perf_counter()
    O.rollout(par, geo, types, s0, cmd, hold, 20, h=0.01)
    per_step = (time.perf_counter() - t) / 20
    steps = int(max(20, min(horizon, target_s / per_step)))
    reps = max(1, int(target_s / (per_step * steps)))
    t = time.perf_counter()
    for _ in range(reps):
        O.rollout(par, geo, types, s0, cmd, hold, steps, h=0.01)
    dt = time.perf_counter() - t
    cores = O.max_threads()
    # one core, on a 512-env slice of the same sample, for the per-core figure
    t1 = time.perf_counter()
    O.rollout(par[:512], geo, types[:512], s0[:512], cmd[:, :512], hold, 100, h=0.01,
              nthreads=1)
    single = 512 * 100 / (time.perf_counter() - t1)
    O.rollout(par[:8], geo, types[:8], s0[:8], cmd[:, :8], hold, 1, h=0.01, nthreads=cores)
    # the small parity fleet: 1,024 nominal BlueROV2 envs, no current, 500 sub-steps
    n1 = 1024
    p1 = np.broadcast_to(nominal[0], (n1, nominal.shape[1])).copy()
    s1 = I.initial_states(21, n1)
    c1 = I.commands(5678, 50, n1, 6).astype(np.float64)
    t1 = time.perf_counter()
    O.rollout(p1, geo, np.zeros(n1, np.int32), s1, c1, hold, 500, h=0.01)
    small = n1 * 500 / (time.perf_counter() - t1)
    return {"value": ns * steps * reps / dt, "unit": "env-steps/s", "cores": cores,
            "kind": "oracle", "single_core_value": single, "small_fleet_value": small,
            "sample": f"{reps}x({ns} envs x {steps} sub-steps), {dt:.1f} s"}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, same metric and workload."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    from oracle import oracle as O
    from paper_2410_14117_gb300 import inputs as I

    vs = I.fleet_vehicles()
    nominal = np.stack([I.round_f32(v.params) for v in vs])
    geo = np.stack([I.round_f32(v.geo()) for v in vs])
    ns = min(args.n_envs, 2048)
    types = np.zeros(ns, dtype=np.int32)
    par = I.round_f32(O.randomize(1234, nominal, types, float(np.float32(0.8)),
                                  float(np.float32(1.2)), float(np.float32(0.2))))
    s0 = I.initial_states(21, ns)
    # size one step to ~0.5 s of host work
    t = time.perf_counter()
    O.rollout(par, geo, types, s0, I.commands(5678, 2, ns, 6).astype(np.float64), args.hold, 20)
    rate = ns * 20 / (time.perf_counter() - t)
    steps = int(max(10, min(args.horizon, 0.5 * rate / ns)))
    cmd = I.commands(5678, math.ceil(steps / args.hold), ns, 6).astype(np.float64)
    for _ in range(args.warmup):
        O.rollout(par, geo, types, s0, cmd, args.hold, steps)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        O.rollout(par, geo, types, s0, cmd, args.hold, steps)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = ns * steps * args.steps / total
    sample = f"{ns} envs x {steps} sub-steps of the headline workload per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "env-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args),
            "cpu_baseline": {"value": value, "unit": "env-steps/s", "cores": O.max_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "env-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def workload_config(args):
    """The headline workload: randomised BlueROV2 envs (parameters U[0.8,1.2] x nominal, NED
    current N(0,0.2)), whole episodes of `horizon` RK4 sub-steps of 0.01 s, commands U[-1,1] held
    `hold` sub-steps; the L2 is flushed (256 MB write, outside the events) between timed
    episodes."""
    return {"workload": f"{args.n_envs} randomised BlueROV2, {args.horizon} RK4 sub-steps",
            "n_envs": args.n_envs, "horizon": args.horizon, "l2": "flushed"}


# ----------------------------------------------------------------------------- our arm

def sig(x, digits=4):
    """x with every float rounded to `digits` significant digits (keeps the JSON line short)."""
    if isinstance(x, float):
        return float(f"{x:.{digits}g}") if math.isfinite(x) else None
    if isinstance(x, dict):
        return {k: sig(v, digits) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [sig(v, digits) for v in x]
    return x


def launch_tag(cfg) -> str:
    """Short name of a launch configuration: schedule/block or chunk/flags."""
    if cfg.schedule == "queue":
        return f"q{cfg.steps_per_launch}w{cfg.warps_per_sm}{'W' if cfg.wide else ''}"
    return f"s{cfg.envs_per_block}k{cfg.steps_per_launch}{'W' if cfg.wide else ''}"


def l2_peak_gbs():
    """The L2's peak bandwidth from profiles/peaks_ncu.txt (ncu: lts__t_bytes.sum.peak_sustained
    bytes per L2 cycle x lts__cycles_elapsed.avg.per_second), or None."""
    path = os.path.join(ROOT, "profiles", "peaks_ncu.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if "l2_gbs" in f:
            return float(f["l2_gbs"])
    return None


def run_ours(args):
    import numpy as np
    import torch

    from paper_2410_14117_gb300 import inputs as I
    from paper_2410_14117_gb300.sim import Sim

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    n, horizon, hold, k = args.n_envs, args.horizon, args.hold, args.k
    vs = I.fleet_vehicles()
    types0 = np.zeros(n, dtype=np.int32)
    if args.no_tune:
        from paper_2410_14117_gb300.autotune import LaunchConfig
        cfg = LaunchConfig("static", args.epb, k)
    else:
        from paper_2410_14117_gb300.autotune import Autotuner
        cfg = Autotuner(horizon=horizon, reps=2).pick(n, types0, vs)
    sim = Sim(n, types0, vs)
    sim.set_env_id_offset(rank_env_offset(rank, n))
    cfg.apply(sim)
    # the fleet is all 6-thruster BlueROV2s: the throttle schedule is stored unpadded,
    # [n_seg][n][6] (24 B per env and segment)
    sim.set_action_width(6)
    n_seg = math.ceil(horizon / hold)
    acts_np = np.ascontiguousarray(I.commands(5678 + rank, n_seg, n, 6)[:, :, :6])
    acts_host = torch.from_numpy(acts_np).pin_memory()
    acts_dev = acts_host.to(dev)
    out_dev = torch.empty((n, 21), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    launches_per_episode = (math.ceil(horizon / cfg.steps_per_launch)
                            if cfg.schedule == "static" else 1)

    # Each episode's parameters are drawn while the previous episode steps
    # (mg_randomize_prefetch on the library's own stream); the episode's mg_randomize installs
    # them with one device copy.
    def episode(seed, a, out):
        sim.randomize(seed, 0.8, 1.2, 0.2, 0.3, wait=False)
        sim.reset()
        sim.set_actions_borrowed(a, hold)  # already resident: read in place
        sim.step(horizon)
        sim.randomize_prefetch(seed + 1)
        sim.get_state(out)

    sim.randomize_prefetch(1000)
    for w in range(max(args.warmup, 3)):
        episode(1000 + w, acts_dev, out_dev)
    torch.cuda.synchronize()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    barrier = (lambda: torch.distributed.barrier()) if world > 1 else (lambda: None)
    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    for i in range(args.steps):
        flush.zero_()
        e0, e1, e2, e3 = ev[i]
        e0.record(stream)
        if i == 0:  # the first timed episode's draw is made inside the timed region too
            sim.randomize_prefetch(2000)
        sim.randomize(2000 + i, 0.8, 1.2, 0.2, 0.3, wait=False)
        sim.reset()
        sim.set_actions_borrowed(acts_dev, hold)
        e1.record(stream)
        sim.step(horizon)
        e2.record(stream)
        sim.randomize_prefetch(2000 + i + 1)
        sim.get_state(out_dev)
        e3.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier()
    clk = clocks.stop()
    assert sim.sync() == 0  # no non-finite state, every mass matrix positive definite
    step_ms = [e[0].elapsed_time(e[3]) for e in ev]
    graph_ms = [e[1].elapsed_time(e[2]) for e in ev]
    total_ms = reduce_max(sum(step_ms), dev)
    value = world * n * horizon * args.steps / (total_ms / 1e3)

    peaks, peak_kind = load_peaks()
    launch_s = statistics.mean(graph_ms) / 1e3 / launches_per_episode
    flops = FLOPS_PER_ENV_STEP[6] * n * horizon / launches_per_episode
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = fp32_alu_peak_tflops(sm_max)
    achieved = flops / launch_s / 1e12
    kname = "k_fleet_queue" if cfg.schedule == "queue" else "k_fleet"
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak,
                "traffic": profiled_traffic(kname, n, horizon // launches_per_episode),
                "kernel": kname, "peak_kind": f"derived ({peak_kind} max SM clock)",
                "flops_per_env_step": FLOPS_PER_ENV_STEP[6], "launch_ms": launch_s * 1e3}

    line = {"metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": dict(workload_config(args), launch=launch_tag(cfg)),
            "roofline": roofline,
            "clocks": clk,
            "gpu_launches": args.steps * (launches_per_episode + 3) + 1}

    # ---- end to end through the C ABI with host buffers: every episode's throttle schedule
    # goes in from page-locked host memory (mg_set_actions_async: the library's copy stream,
    # one of two device buffers, overlapping the previous episode's steps) and every episode's
    # final state comes back to page-locked host memory (mg_get_state_async: the library's
    # read-back stream, overlapping the next episode); each episode's parameters are drawn
    # while the previous episode steps (mg_randomize_prefetch) and installed without a host wait
    # (MG_RANDOMIZE_ASYNC: the fleet's mass matrices are diagonal).  All copies and draws have
    # completed when the clock stops (mg_sync).  50 episodes back to back, pipeline fill
    # included.
    if not args.no_e2e:
        ke = min(args.steps, 50)
        outs_host = [torch.empty((n, 21), dtype=torch.float32).pin_memory() for _ in range(2)]

        def e2e_episodes(count, seed0):
            sim.randomize_prefetch(seed0)
            for i in range(count):
                sim.set_actions_async(acts_host, hold)
                sim.randomize(seed0 + i, 0.8, 1.2, 0.2, 0.3, wait=False)
                sim.reset()
                sim.step(horizon)
                sim.randomize_prefetch(seed0 + i + 1)
                sim.get_state_async(outs_host[i % 2])
            assert sim.sync() == 0

        e2e_episodes(2, 1)
        barrier()
        t = time.perf_counter()
        e2e_episodes(ke, 3000)
        el = reduce_max(time.perf_counter() - t, dev)
        line["e2e"] = {"value": world * n * horizon * ke / el, "unit": "env-steps/s",
                       "h2d_bytes_per_step": acts_np.nbytes,
                       "d2h_bytes_per_step": n * 21 * 4}

    # ---- the plain per-step form on the same GPU (one launch per sub-step)
    if not args.no_per_step:
        fused_ms = statistics.mean(graph_ms)
        ps = bench_per_step(sim, acts_dev, args, peaks, peak_kind)
        host_ms, ps_ms, k50_ms = ps.pop("host_ms"), ps.pop("graph_ms"), ps.pop("k50_ms")
        # the autotuned persistent form, and the static k = 50 form in one CUDA graph, over the
        # per-step form launched from the host and replayed from a graph
        line["fused_over_per_step"] = {"host": host_ms / fused_ms, "graph": ps_ms / fused_ms,
                                       "k50_over_host": host_ms / k50_ms,
                                       "k50_over_graph": ps_ms / k50_ms}
        line["per_step"] = ps
        cfg.apply(sim)

    sim.close()
    if not args.no_per_step and world == 1:
        line["per_step"]["1M"] = bench_per_step_large(vs, args, peaks, peak_kind)
    if not args.no_extra and world == 1:
        line["small_fleet"] = bench_small_fleet(vs)
        line["size_sweep"] = bench_size_sweep(vs)
        line["mixed_fleet"] = bench_mixed_fleet(vs)
        line["adjoint"] = bench_adjoint(vs)
        line["task"] = bench_task(vs)
        line["env"] = bench_env()
        line["split"] = bench_split(vs)
        line["full_hydro"] = bench_full_hydro(vs)
        line["serve"] = bench_serve(vs, args.serve_seconds)

    if world == 1 and rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(n, horizon, hold)

    if rank == 0:
        print(json.dumps(sig(line), separators=(",", ":")), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ----------------------------------------------------------------------------- other configs

def _time_episodes(fn, reps):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _per_step_roofline(bytes_per_launch, launch_s, n, bound, peak, peak_kind, traffic):
    ach = bytes_per_launch / launch_s / 1e9
    return {"bound": bound, "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak if peak else None,
            "peak_kind": peak_kind, "bytes_per_env_step": bytes_per_launch // n,
            "launch_us": launch_s * 1e6, "traffic": traffic}


def bench_per_step(sim, acts_dev, args, peaks, peak_kind):
    """The headline fleet (65,536 envs) in the plain per-step form: one static-grid launch per
    sub-step (128-register kernel, 16 warps/SM), host-launched and replayed from one CUDA graph,
    and the persistent form as the scale configuration names it (static grid, 50 sub-steps per
    launch, one graph).  Its working set (state, parameters, one command: 20 MB) stays in the
    129 MB L2 from launch to launch (ncu, steady state: no DRAM reads, ~40 KB of DRAM writes
    against 25 MB of L2 traffic per launch), so its roofline is the L2's bandwidth (ncu's peak),
    not HBM; it runs far below it (launch- and latency-bound)."""
    import torch
    n, horizon, hold = args.n_envs, args.horizon, args.hold
    stream = torch.cuda.current_stream()
    sim.set_actions_borrowed(acts_dev, hold)
    sim.set_schedule(False, False)
    sim.set_launch(args.epb, 1, False)
    sim.randomize(7, 0.8, 1.2, 0.2, 0.3)
    sim.reset()
    for _ in range(50):
        sim.step(1)
    reps = 2
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def host_loop():
        sim.set_actions_borrowed(acts_dev, hold)
        for _ in range(horizon):
            sim.step(1)

    def graph_episode():
        sim.set_actions_borrowed(acts_dev, hold)
        sim.step(horizon)

    host_ms = timed(host_loop)
    sim.set_launch(args.epb, 1, True)
    graph_episode()  # capture
    graph_ms = timed(graph_episode)
    sim.set_launch(args.epb, 50, True)
    graph_episode()  # capture
    k50_ms = timed(graph_episode)
    launch_s = graph_ms / 1e3 / horizon
    bytes_per_launch = n * (2 * STATE_BYTES[6] + PARAM_BYTES + CMD_BYTES[6])
    l2 = l2_peak_gbs()
    return {"host": n * horizon / (host_ms / 1e3), "graph": n * horizon / (graph_ms / 1e3),
            "k50_graph": n * horizon / (k50_ms / 1e3),
            "roofline": _per_step_roofline(bytes_per_launch, launch_s, n, "l2", l2,
                                           "ncu L2 peak", profiled_traffic("k_fleet_step1", n, 1)),
            "host_ms": host_ms, "graph_ms": graph_ms, "k50_ms": k50_ms}


def bench_per_step_large(vs, args, peaks, peak_kind, n=1 << 20, steps=200):
    """The per-step form where its working set (312 MB per launch) is well past the L2: a
    1,048,576-env randomised BlueROV2 fleet, one launch per sub-step replayed from a CUDA graph,
    unpadded buffered commands; bounded by HBM bandwidth."""
    import numpy as np
    import torch
    from paper_2410_14117_gb300 import inputs as I
    from paper_2410_14117_gb300.sim import Sim

    sim = Sim(n, np.zeros(n, np.int32), vs)
    sim.set_schedule(False, False)
    sim.set_launch(args.epb, 1, True)
    sim.set_action_width(6)
    sim.randomize(8, 0.8, 1.2, 0.2, 0.3)
    sim.reset()
    acts = torch.tensor(np.ascontiguousarray(I.commands(9, steps // args.hold, n, 6)[:, :, :6]),
                        device="cuda")

    def episode():
        sim.set_actions_borrowed(acts, args.hold)
        sim.step(steps)

    ms = _time_episodes(episode, 3)
    assert sim.sync() == 0
    # the persistent form on the same fleet, for the ratio at this size (200-register static grid)
    sim.set_schedule(False, True)
    sim.set_launch(64, 1000, True)
    fused_ms = _time_episodes(episode, 3)
    sim.close()
    launch_s = ms / 1e3 / steps
    bytes_per_launch = n * (2 * STATE_BYTES[6] + PARAM_BYTES + CMD_BYTES[6])
    return {"graph": n * steps / (ms / 1e3), "fused_over_graph": ms / fused_ms,
            "roofline": _per_step_roofline(bytes_per_launch, launch_s, n, "hbm",
                                           float(peaks.get("hbm_gbs", 6800.0)),
                                           f"{peak_kind} hbm_gbs",
                                           profiled_traffic("k_fleet_step1", n, 1))}


def bench_small_fleet(vs, n=1024, horizon=500, reps=5):
    """The small parity fleet: 1,024 nominal BlueROV2 envs, no current, commands U[-1,1] held
    10 sub-steps, 500 sub-steps of 0.01 s (parity against the oracle is in the tests)."""
    import numpy as np
    import torch
    from paper_2410_14117_gb300 import inputs as I
    from paper_2410_14117_gb300.autotune import Autotuner
    from paper_2410_14117_gb300.sim import Sim

    types = np.zeros(n, np.int32)
    sim = Sim(n, types, vs)
    launch = Autotuner(horizon=horizon, reps=2).tune(sim, vs)
    acts = torch.tensor(I.commands(5678, horizon // 10, n, 6), device="cuda")
    s0 = torch.tensor(I.initial_states(21, n), dtype=torch.float32, device="cuda")

    def episode():
        sim.set_state(s0)
        sim.set_actions_borrowed(acts, 10)
        sim.step(horizon)

    ms = _time_episodes(episode, reps)
    sim.close()
    return {"rate": n * horizon / (ms / 1e3), "launch": launch_tag(launch)}


def bench_size_sweep(vs, sizes=(4096, 16384, 65536, 262144, 1048576), horizon=1000, reps=3):
    """Config-2 sweep: the headline workload's sub-steps (randomised BlueROV2, current,
    procedural commands held 10) at each fleet size, with the launch the autotuner picks for
    that size.  Rows [envs, env-sub-steps/s, fraction of the FP32 ALU peak, launch]."""
    import numpy as np
    from paper_2410_14117_gb300.autotune import Autotuner
    from paper_2410_14117_gb300.sim import Sim

    peak = fp32_alu_peak_tflops(2070.0)
    tuner = Autotuner(horizon=horizon, reps=2)
    rows = []
    for n in sizes:
        types = np.zeros(n, np.int32)
        cfg = tuner.pick(n, types, vs)
        sim = Sim(n, types, vs)
        cfg.apply(sim)
        sim.randomize(1234, 0.8, 1.2, 0.2, 0.3)
        sim.reset()
        sim.set_procedural_actions(5678, 10)
        ms = _time_episodes(lambda: sim.step(horizon), reps)
        assert sim.sync() == 0
        sim.close()
        rate = n * horizon / (ms / 1e3)
        rows.append([n, rate, rate * FLOPS_PER_ENV_STEP[6] / (peak * 1e12), launch_tag(cfg)])
    return rows


def bench_mixed_fleet(vs, n=262144, horizon=500, reps=5):
    """Mixed BlueROV2 / BlueROV2-Heavy fleet, groups log-uniform in [1, 32768] (60/40 types),
    randomised; autotuned launch; against a homogeneous BlueROV2 fleet of the same size."""
    import numpy as np
    from paper_2410_14117_gb300 import inputs as I
    from paper_2410_14117_gb300.autotune import Autotuner
    from paper_2410_14117_gb300.sim import Sim

    out = {}
    tuner = Autotuner(horizon=horizon, reps=2)
    for name, types in (("mixed", I.mixed_fleet(3, n)), ("homog", np.zeros(n, np.int32))):
        cfg = tuner.pick(n, types, vs)
        sim = Sim(n, types, vs)
        cfg.apply(sim)
        sim.randomize(1234, 0.8, 1.2, 0.2, 0.3)
        sim.reset()
        sim.set_procedural_actions(5678, 10)
        ms = _time_episodes(lambda: sim.step(horizon), reps)
        assert sim.sync() == 0
        out[name] = n * horizon / (ms / 1e3)
        out[name + "_launch"] = launch_tag(cfg)
        if name == "mixed":
            out["groups"] = int(np.count_nonzero(np.diff(types)) + 1)
            out["heavy_frac"] = float((types == 1).mean())
        sim.close()
    out["ratio"] = out["mixed"] / out["homog"]
    return out


def bench_adjoint(vs, n=4096, T=200, C=20, reps=5):
    """Differentiable rollout: forward (recording + checkpoints) and hand-written adjoint,
    4,096 BlueROV2 envs, 200 sub-steps, checkpoints every 20, MSE on the trajectory."""
    import numpy as np
    import torch
    from paper_2410_14117_gb300 import inputs as I
    from paper_2410_14117_gb300.adjoint import COEF_SLICE, rollout
    from paper_2410_14117_gb300.autotune import Autotuner
    from paper_2410_14117_gb300.sim import Sim

    sim = Sim(n, np.zeros(n, np.int32), vs)
    # the forward's checkpoint segments are launches of C sub-steps: tune for that call size
    Autotuner(horizon=T, reps=2, k_per_call=C).tune(sim, vs)
    sim.randomize(1234, 0.8, 1.2, 0.2, 0.3)
    params = sim.get_params()
    coeffs = params[:, COEF_SLICE].clone().requires_grad_(True)
    acts = torch.tensor(I.commands(5678, T // 10, n, 6), device="cuda", requires_grad=True)
    s0 = torch.tensor(I.initial_states(21, n), dtype=torch.float32, device="cuda")
    target = torch.zeros((T, n, 13), device="cuda")

    def fwd():
        return rollout(sim, coeffs, acts, s0, 10, T, C)

    f_ms = _time_episodes(fwd, reps)

    def fb():
        tr = rollout(sim, coeffs, acts, s0, 10, T, C)
        return torch.autograd.grad(((tr - target) ** 2).mean(), (coeffs, acts))

    fb_ms = _time_episodes(fb, reps)  # backward kernel chosen by fleet size
    sim.set_adjoint_mode(1)            # one warp per 32 envs, for comparison
    fb1_ms = _time_episodes(fb, reps)
    sim.set_adjoint_mode(0)
    sim.close()
    return {"fwd_ms": f_ms, "fwd_bwd_ms": fb_ms, "bwd_over_fwd": (fb_ms - f_ms) / f_ms,
            "fwd_bwd_1warp_ms": fb1_ms}


def bench_task(vs, n=65536, k=10, steps=100, reps=3):
    """Task layer (§EXPERIMENTS): circle tracking with 3 look-ahead points, auto-reset, one task
    step = k sub-steps + observation (Eq. 2) + error (Eq. 4); against plain stepping."""
    import numpy as np
    import torch
    from paper_2410_14117_gb300.autotune import Autotuner
    from paper_2410_14117_gb300.sim import Sim

    types = np.zeros(n, np.int32)
    sim = Sim(n, types, vs)
    Autotuner(horizon=k * 10, reps=2, k_per_call=k).tune(sim, vs)
    sim.randomize(11, 0.8, 1.2, 0.2, 0.3)
    sim.reset()
    sim.set_procedural_actions(12, k)
    # each env spawns (at the origin) within 0.5 m of its circle's starting point
    g = np.random.default_rng(5)
    phase = g.uniform(0.0, 2 * np.pi, n)
    centres = np.zeros((n, 4))
    centres[:, 0] = -2.0 * np.cos(phase)
    centres[:, 1] = -2.0 * np.sin(phase)
    centres[:, :3] += g.uniform(-0.5, 0.5, (n, 3)) / np.sqrt(3.0)
    centres[:, 3] = phase
    centres = torch.tensor(centres, dtype=torch.float32, device="cuda")
    sim.set_task(1, centres, radius=2.0, omega=0.4, vz=0.0, lookahead=3, lookahead_dt=0.5,
                 max_error=3.0, episode_steps=1000)

    def loop():
        for _ in range(steps):
            sim.task_step(k)

    def plain():
        for _ in range(steps):
            sim.step(k)

    task_ms = _time_episodes(loop, reps)
    resets = _count_resets(sim, k, steps)
    plain_ms = _time_episodes(plain, reps)
    observe_ms = _time_episodes(lambda: [sim.task_step(0) for _ in range(steps)], reps)
    sim.close()
    return {"rate": n * k * steps / (task_ms / 1e3), "plain": n * k * steps / (plain_ms / 1e3),
            "step_us": task_ms / steps * 1e3, "observe_us": observe_ms / steps * 1e3,
            "resets": resets}


def bench_env(sizes=(4096, 65536), k=10, steps=100, reps=3):
    """The Gym-style environment (MarineEnv, §EXPERIMENTS' task format): BlueROV2 Heavy circle
    tracking, one throttle vector per env and step held over k sub-steps, the actions copied
    in by the step call; rows [envs, µs per env step, env-sub-steps/s]."""
    import torch
    from paper_2410_14117_gb300.env import MarineEnv

    rows = []
    for n in sizes:
        env = MarineEnv(n, task="circle", vehicle=1, sub_steps=k, seed=3)
        g = torch.Generator(device="cuda").manual_seed(5)
        acts = torch.rand((steps, n, env.action_dim), generator=g, device="cuda") * 2 - 1
        env.reset()

        def loop():
            for i in range(steps):
                env.step(acts[i])

        ms = _time_episodes(loop, reps)
        env.close()
        rows.append([n, ms / steps * 1e3, n * k * steps / (ms / 1e3)])
    return rows


def _count_resets(sim, k, steps):
    n_done = 0
    for _ in range(steps):
        n_done += int(sim.task_step(k)[2].sum())
    return n_done / steps


def bench_split(vs, n=65536, horizon=1000, n_acc=4096, reps=3):
    """The paper's split integration (§METHOD: engine-integrated rigid body, hydrodynamic term
    as an external force with the previous sub-step's acceleration in its added-mass part)
    against the coupled RK4 step: throughput, accuracy at h = 0.01 against the coupled equation
    at h = 0.001 (4,096 envs, added mass halved so that it is stable, 1 s), and the share of
    randomised envs the lagged added mass destabilises."""
    import numpy as np
    import torch
    from paper_2410_14117_gb300 import inputs as I
    from paper_2410_14117_gb300.sim import Sim

    def fleet(n_envs, seed, ma_scale, sigma=0.3):
        sim = Sim(n_envs, np.zeros(n_envs, np.int32), vs)
        sim.randomize(seed, 0.8, 1.2, 0.2, sigma)
        if ma_scale != 1.0:
            p = sim.get_params()
            p[:, I.P_MA:I.P_MA + 6] *= ma_scale
            sim.set_params(p)
        sim.reset()
        return sim

    out = {}
    # throughput, added mass halved so that every env stays finite
    sim = fleet(n, 1234, 0.5)
    sim.set_launch(128, horizon, False)
    sim.set_procedural_actions(5678, 10)
    acc = torch.zeros((6, n), device="cuda")
    split_ms = _time_episodes(lambda: sim.step_split(horizon, acc), reps)
    sim.set_launch(128, 50, True)
    coupled_ms = _time_episodes(lambda: sim.step(horizon), reps)
    sim.close()
    out["split"] = n * horizon / (split_ms / 1e3)
    out["coupled"] = n * horizon / (coupled_ms / 1e3)
    # the general form: off-centre gravity (r_g ~ U[-2, 2] cm), 10 %-coupled M_A and D_l
    sim = Sim(n, np.zeros(n, np.int32), vs)
    sim.randomize(1234, 0.8, 1.2, 0.2, 0.3, rg_halfwidth=0.02)
    p = sim.get_params()
    p[:, I.P_MA:I.P_MA + 6] *= 0.4
    sim.set_params(p)
    sim.set_hydro_offdiag(torch.tensor(I.hydro_offdiag(9, p.double().cpu().numpy(), 0.1),
                                       dtype=torch.float32, device="cuda"))
    sim.reset()
    sim.set_launch(128, horizon, False)
    sim.set_procedural_actions(5678, 10)
    acc.zero_()
    general_ms = _time_episodes(lambda: sim.step_split(horizon, acc), reps)
    sim.close()
    out["split_general"] = n * horizon / (general_ms / 1e3)
    # accuracy: the same commands in time (held 0.1 s) at h = 0.01 and the h = 0.001 reference
    res = {}
    for name, dt, hold, steps, split in (("ref", 0.001, 100, 1000, False),
                                         ("coupled", 0.01, 10, 100, False),
                                         ("split", 0.01, 10, 100, True)):
        sim = fleet(n_acc, 77, 0.5)
        sim.set_timestep(dt)
        sim.set_procedural_actions(88, hold)
        if split:
            sim.step_split(steps, torch.zeros((6, n_acc), device="cuda"))
        else:
            sim.step(steps)
        res[name] = sim.get_state().double().cpu().numpy()
        sim.close()
    for name in ("coupled", "split"):
        dp = np.abs(res[name][:, 0:3] - res["ref"][:, 0:3]).max(axis=1)
        out[f"{name}_pos_err_m"] = [float(np.median(dp)), float(dp.max())]
    # stability with the randomised nominal added mass
    sim = fleet(n_acc, 99, 1.0)
    p = sim.get_params().double().cpu().numpy()
    ratio = np.concatenate([p[:, I.P_MA:I.P_MA + 3] / p[:, [I.P_M]],
                            p[:, I.P_MA + 3:I.P_MA + 6] / p[:, I.P_IG:I.P_IG + 3]], axis=1)
    sim.set_procedural_actions(5, 10)
    sim.step_split(1000, torch.zeros((6, n_acc), device="cuda"))
    st = sim.get_state().double().cpu().numpy()
    sim.close()
    blown = ~np.isfinite(st).all(axis=1) | (np.abs(st[:, 7:13]).max(axis=1) > 100.0)
    out["unstable_pred"] = float((ratio.max(axis=1) > 1.0).mean())
    out["diverged"] = float(blown.mean())
    return out


def bench_full_hydro(vs, n=65536, horizon=1000, reps=3):
    """Full (non-diagonal) added mass and linear damping with randomised centres of gravity
    (r_g ~ U[-2, 2] cm per axis, off-diagonal M_A and D_l at 15 % coupling): the general path
    with the off-diagonal coefficients staged per block, against the diagonal-mass path, same
    fleet size and workload."""
    import numpy as np
    import torch
    from paper_2410_14117_gb300 import inputs as I
    from paper_2410_14117_gb300.sim import Sim

    out = {}
    for name in ("diag", "full", "full_queue"):
        sim = Sim(n, np.zeros(n, np.int32), vs)
        sim.set_launch(128, horizon, True)
        if name == "full_queue":  # the work-queue schedule's off-diagonal variant, chunk 100
            sim.set_launch(128, 100, True)
            sim.set_schedule(True, True, 8)
        if name != "diag":
            sim.randomize(1234, 0.8, 1.2, 0.2, 0.3, rg_halfwidth=0.02)
            p = sim.get_params().double().cpu().numpy()
            sim.set_hydro_offdiag(torch.tensor(I.hydro_offdiag(9, p), dtype=torch.float32,
                                               device="cuda"))
        else:
            sim.randomize(1234, 0.8, 1.2, 0.2, 0.3)
        sim.reset()
        sim.set_procedural_actions(5678, 10)
        ms = _time_episodes(lambda: sim.step(horizon), reps)
        assert sim.sync() == 0
        sim.close()
        out[name] = n * horizon / (ms / 1e3)
    out["ratio"] = max(out["full"], out["full_queue"]) / out["diag"]
    return out


# Sub-steps per serving tick: at 200 req/s p50 / p99 were 0.73 / 2.06 ms with 50, 0.67 / 2.08
# with 100 and 0.64 / 2.01 with 200 (Python request loop); at 2,000 req/s 100 cut p99 from 6.5
# to 6.0 ms.
SERVE_K = 100


def bench_serve(vs, seconds, rate=200.0):
    """Poisson arrivals of rollout jobs (envs log-uniform [64, 65536], horizon U[50, 1000],
    type 50/50, randomised parameters and currents, trajectory recorded) served with continuous
    batching under a 120 GB budget by the native request loop (mg_server_*), and the same stream
    served one job at a time; each server first serves one second of the same job mix (its
    record memory pool warm), as the measured stream's own arrivals would after a while.  Then
    the same job mix at 10x the arrival rate."""
    from paper_2410_14117_gb300 import inputs as I
    from paper_2410_14117_gb300.serve import NativeServer, Server, requests_from_specs

    specs = I.serving_jobs(42, seconds, rate_hz=rate)
    out = {"jobs": len(specs)}
    keys = ("p50_ms", "p99_ms", "env_steps_per_s")
    for mode in ("batched", "serial"):
        srv = NativeServer(vs, budget_bytes=120e9, capacity_envs=8 << 20, k=SERVE_K)
        srv.run(requests_from_specs(I.serving_jobs(7, 1.0, rate_hz=rate)), mode=mode)
        _, st = srv.run(requests_from_specs(specs), mode=mode)
        srv.close()
        out[mode] = [st[k] for k in keys]
    # the same stream through the Python request loop (Server), batched
    srv = Server(vs, budget_bytes=120e9, capacity_envs=8 << 20, k=SERVE_K)
    srv.run(requests_from_specs(I.serving_jobs(7, 1.0, rate_hz=rate)), mode="batched")
    _, st = srv.run(requests_from_specs(specs), mode="batched")
    srv.close()
    out["python_batched"] = [st[k] for k in keys]
    hot = I.serving_jobs(43, seconds / 4, rate_hz=10 * rate)
    out["stress_jobs"] = len(hot)
    for mode in ("batched", "serial"):
        srv = NativeServer(vs, budget_bytes=120e9, capacity_envs=8 << 20, k=SERVE_K)
        srv.run(requests_from_specs(I.serving_jobs(8, seconds / 4, rate_hz=10 * rate)),
                mode=mode)
        _, st = srv.run(requests_from_specs(hot), mode=mode)
        srv.close()
        out["stress_" + mode] = [st[k] for k in keys]
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
