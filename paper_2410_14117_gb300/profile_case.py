"""A small, self-contained workload for profiling the step kernel under ncu.

    python -m paper_2410_14117_gb300.profile_case --n-envs 65536 --k 50 --launches 3

Builds a domain-randomised BlueROV2 fleet with NED current and a buffered throttle schedule
(commands U[-1,1] held 10 sub-steps), then issues ``launches`` calls of ``mg_step(k)`` (no CUDA graph)
after a few warm-up calls: with ``--static`` each is one launch of the static-grid kernel running
``k`` sub-steps; otherwise each is one work-queue launch covering ``k`` sub-steps in chunks of
``--chunk``; with ``--task`` each is one circle-tracking task step (``k`` sub-steps and the fused
observation / error / auto-reset epilogue, static grid); ``--split`` runs the split-integration
comparison kernel, ``--full`` the general path with off-diagonal hydrodynamics; ``--adjoint`` runs
``launches`` forward and backward passes of the differentiable rollout (``k`` sub-steps,
checkpoints every ``--chunk``, MSE loss on the trajectory; ``--adjoint-mode`` picks the backward
kernel; with ``--full`` on the general path); ``--serve JOBS`` runs ``launches`` serving ticks of ``k`` sub-steps over JOBS jobs in a
job pool.  Holds well under a GB of device
memory at 65,536 envs.
"""
from __future__ import annotations

import argparse
import math

import numpy as np
import torch

from . import inputs as I
from .sim import Sim


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-envs", type=int, default=65536)
    ap.add_argument("--k", type=int, default=50)
    ap.add_argument("--chunk", type=int, default=50)
    ap.add_argument("--launches", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--epb", type=int, default=128)
    ap.add_argument("--vehicle", type=int, default=0)
    ap.add_argument("--static", action="store_true",
                    help="static grid (one launch per k sub-steps) instead of the work queue")
    ap.add_argument("--narrow", action="store_true",
                    help="the 128-register diagonal-mass kernel instead of the 200-register one "
                         "(work queue; static grid)")
    ap.add_argument("--wps", type=int, default=8, help="work queue: resident warps per SM cap")
    ap.add_argument("--width6", action="store_true",
                    help="unpadded throttle schedule, 6 floats per env and segment "
                         "(mg_set_action_width; 6-thruster vehicle)")
    ap.add_argument("--task", action="store_true",
                    help="circle-tracking task steps of k sub-steps (fused task epilogue) instead "
                         "of plain steps; static grid")
    ap.add_argument("--split", action="store_true",
                    help="split-integration comparison steps (mg_step_split), added mass halved")
    ap.add_argument("--full", action="store_true",
                    help="off-diagonal added mass and damping, r_g ~ U[-2, 2] cm (general path, "
                         "static grid)")
    ap.add_argument("--adjoint", action="store_true",
                    help="forward + backward passes of the differentiable rollout instead")
    ap.add_argument("--serve", type=int, default=0, metavar="JOBS",
                    help="serving ticks instead: JOBS jobs of n_envs / JOBS envs each (types "
                         "alternating BlueROV2 / Heavy) in a job pool, each launch one tick of k "
                         "sub-steps over all of them")
    ap.add_argument("--adjoint-mode", type=int, default=0,
                    help="backward kernel (mg_set_adjoint_mode): 0 by size, 1 one warp, 2 two warps")
    args = ap.parse_args()
    if args.adjoint:
        return adjoint_case(args)
    if args.serve:
        return serve_case(args)

    n = args.n_envs
    vs = I.fleet_vehicles()
    sim = Sim(n, np.full(n, args.vehicle, dtype=np.int32), vs)
    sim.set_launch(args.epb, args.k if args.static else args.chunk, False)
    sim.set_schedule(not args.static, not args.narrow, args.wps)
    sim.randomize(1234, 0.8, 1.2, 0.2, 0.3, rg_halfwidth=0.02 if args.full else 0.0)
    if args.split:
        p = sim.get_params()
        p[:, I.P_MA:I.P_MA + 6] *= 0.5
        sim.set_params(p)
    if args.full:
        p = sim.get_params().double().cpu().numpy()
        sim.set_hydro_offdiag(torch.tensor(I.hydro_offdiag(9, p), dtype=torch.float32,
                                           device="cuda"))
    sim.reset()
    acc = torch.zeros((6, n), device="cuda") if args.split else None
    total = (args.warmup + args.launches) * args.k
    cmds = I.commands(5678, math.ceil(total / 10), n, vs[args.vehicle].n_thr)
    if args.width6:
        sim.set_action_width(6)
        cmds = np.ascontiguousarray(cmds[:, :, :6])
    sim.set_actions(torch.tensor(cmds, device="cuda"), 10)
    if args.task:
        sim.set_schedule(False)
        g = np.random.default_rng(5)
        phase = g.uniform(0.0, 2 * np.pi, n)
        centres = np.c_[-2.0 * np.cos(phase), -2.0 * np.sin(phase), np.zeros(n), phase]
        sim.set_task(1, torch.tensor(centres, dtype=torch.float32, device="cuda"), radius=2.0,
                     omega=0.4, lookahead=3, lookahead_dt=0.5, max_error=3.0,
                     episode_steps=1000)
    for _ in range(args.warmup + args.launches):
        if args.task:
            sim.task_step(args.k)
        elif args.split:
            sim.step_split(args.k, acc)
        else:
            sim.step(args.k)
    bad = sim.sync()
    sim.close()
    print(f"profile_case: {n} envs, {args.launches} launches of k={args.k}, non-finite {bad}")


def adjoint_case(args):
    from .adjoint import COEF_SLICE, rollout

    n, T, C = args.n_envs, args.k, args.chunk
    vs = I.fleet_vehicles()
    sim = Sim(n, np.full(n, args.vehicle, dtype=np.int32), vs)
    sim.set_launch(args.epb, 1000, True)
    sim.set_adjoint_mode(args.adjoint_mode)
    sim.randomize(1234, 0.8, 1.2, 0.2, 0.3, rg_halfwidth=0.02 if args.full else 0.0)
    if args.full:  # the general path: off-centre gravity and the off-diagonal extension
        p = sim.get_params().double().cpu().numpy()
        sim.set_hydro_offdiag(torch.tensor(I.hydro_offdiag(9, p), dtype=torch.float32,
                                           device="cuda"))
    coeffs = sim.get_params()[:, COEF_SLICE].clone().requires_grad_(True)
    acts = torch.tensor(I.commands(5678, math.ceil(T / 10), n, vs[args.vehicle].n_thr),
                        device="cuda", requires_grad=True)
    s0 = torch.tensor(I.initial_states(21, n), dtype=torch.float32, device="cuda")
    for _ in range(args.warmup + args.launches):
        traj = rollout(sim, coeffs, acts, s0, 10, T, C)
        grads = torch.autograd.grad((traj ** 2).mean(), (coeffs, acts))
    torch.cuda.synchronize()
    sim.close()
    print(f"profile_case: adjoint, {n} envs, T={T}, C={C}, |dL/dcoef|_1 "
          f"{float(grads[0].abs().sum()):.4e}")


def serve_case(args):
    from .serve import Pool

    vs = I.fleet_vehicles()
    per = args.n_envs // args.serve
    pool = Pool(per * args.serve, vs)
    horizon = args.k * (args.warmup + args.launches)
    for j in range(args.serve):
        jid = pool.admit(per, j % 2, horizon, 100 + j, 200 + j, hold=10)
        assert jid is not None
    for _ in range(args.warmup + args.launches):
        pool.tick(args.k)
    pool.sync()
    print(f"profile_case: serve, {args.serve} jobs x {per} envs, "
          f"{args.warmup + args.launches} ticks of k={args.k}")


if __name__ == "__main__":
    main()
