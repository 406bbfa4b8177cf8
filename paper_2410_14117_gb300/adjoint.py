"""Differentiable rollout: ``RolloutFn`` (a ``torch.autograd.Function``) advances a fleet T RK4
sub-steps with given hydrodynamic coefficients and throttle actions and returns the trajectory;
its backward is the hand-written discrete adjoint in libmg.so (mg_rollout_backward), checkpointed
every C sub-steps.  Gradients flow to the per-env coefficients (added-mass, linear and quadratic
damping diagonals of Eq. 1) and to every action segment (Eq. 3)."""
from __future__ import annotations

import ctypes
import math

import torch

from ._lib import MG_MAX_THR, MG_NPARAM, MG_NSTATE, MG_NTRAJ, call
from .sim import Sim, _ptr

NCOEF = 18
COEF_SLICE = slice(4, 22)  # parameter-record entries of M_A, Dl, Dq


class RolloutFn(torch.autograd.Function):
    """traj = RolloutFn.apply(sim, coeffs, actions, state0, hold, T, C)

    coeffs [n, 18] float32 (device), actions [n_seg, n, 8] float32 (device), state0 [n, 21].
    Returns traj [T, n, 13]: (p, q, nu) after every sub-step.  The sim's other parameters are
    kept; its state after the call is the rollout's final state."""

    @staticmethod
    def forward(ctx, sim: Sim, coeffs, actions, state0, hold: int, T: int, C: int = 20):
        n = sim.n
        params = sim.get_params()
        params[:, COEF_SLICE] = coeffs.to(torch.float32)
        sim.set_params(params.contiguous())
        sim.set_state(state0.to(torch.float32).contiguous())
        acts = actions.to(torch.float32).contiguous()
        sim.set_actions(acts, hold)
        traj = torch.empty((T, MG_NTRAJ, n), dtype=torch.float32, device=sim.device)
        ckpt = torch.empty((math.ceil(T / C), MG_NSTATE, n), dtype=torch.float32,
                           device=sim.device)
        step0 = ctypes.c_int64()
        call("mg_rollout_forward", sim._h, int(T), int(C), _ptr(traj), _ptr(ckpt),
             ctypes.byref(step0))
        ctx.sim, ctx.T, ctx.C, ctx.step0 = sim, T, C, step0.value
        ctx.act_shape = acts.shape
        ctx.save_for_backward(ckpt)
        return traj.permute(0, 2, 1)

    @staticmethod
    def backward(ctx, g):
        (ckpt,) = ctx.saved_tensors
        sim = ctx.sim
        dtraj = g.permute(0, 2, 1).contiguous().to(torch.float32)
        dcoef = torch.empty((sim.n, NCOEF), dtype=torch.float32, device=sim.device)
        dact = torch.zeros(ctx.act_shape, dtype=torch.float32, device=sim.device)
        dstate0 = torch.empty((sim.n, MG_NSTATE), dtype=torch.float32, device=sim.device)
        call("mg_rollout_backward", sim._h, int(ctx.T), int(ctx.C), _ptr(ckpt), _ptr(dtraj),
             int(ctx.step0), _ptr(dcoef), _ptr(dact), _ptr(dstate0))
        return None, dcoef, dact, dstate0, None, None, None


def rollout(sim: Sim, coeffs, actions, state0, hold: int, T: int, C: int = 20):
    """Differentiable trajectory [T, n, 13] (see RolloutFn)."""
    return RolloutFn.apply(sim, coeffs, actions, state0, hold, T, C)


def shared_coefficient_grad(dcoef, group=None):
    """Gradient with respect to coefficients shared by every env of every rank (one set of 18
    for the whole sharded fleet, e.g. when identifying a vehicle model from many runs): the sum
    of the per-env gradients ``dcoef`` [n_local, 18] over this rank's envs, summed over the ranks
    of ``group`` by one all-reduce of 18 FP32 values — the only collective of the sharded path.
    Without an initialised process group it is the local sum."""
    local = dcoef.sum(dim=0)
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.all_reduce(local, op=torch.distributed.ReduceOp.SUM, group=group)
    return local
