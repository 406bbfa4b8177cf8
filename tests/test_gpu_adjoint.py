"""Hand-written discrete adjoint of the rollout (libmg.so, through RolloutFn) against central
finite differences of the FP64 oracle's rollout: gradients of a trajectory MSE with respect to
the 18 hydrodynamic coefficients of every env and to every buffered action, relative error
<= 1e-3 per env."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2410_14117_gb300 import inputs as I
from paper_2410_14117_gb300.adjoint import COEF_SLICE, rollout
from paper_2410_14117_gb300.sim import MGError, Sim

from _helpers import f32, oracle_geo, oracle_nominal, vehicles

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-3
FD_REL = 1e-6


def _problem(n=64, T=200, hold=10, seed=0, vehicle=0):
    vs = vehicles()
    types = np.full(n, vehicle, dtype=np.int32)
    nt = vs[vehicle].n_thr
    params = I.round_f32(O.randomize(1234 + seed, oracle_nominal(vs), types, f32(0.8), f32(1.2),
                                     f32(0.2)))
    s0 = I.initial_states(21 + seed, n)
    cmds = I.commands(5678 + seed, T // hold, n, nt).astype(np.float64)
    # target: the same start and commands with coefficients x U[0.9, 1.1]
    g = np.random.default_rng(99 + seed)
    pt = params.copy()
    pt[:, COEF_SLICE] *= g.uniform(0.9, 1.1, size=(n, 18))
    pt = I.round_f32(pt)
    _, target = O.rollout(pt, oracle_geo(vs), types, s0, cmds, hold, T, record=True)
    target = I.round_f32(target[:, :, :13])  # [T, n, 13]
    return vs, types, params, s0, cmds, target


def _oracle_losses(vs, types, params, s0, cmds, target, hold, T):
    _, traj = O.rollout(params, oracle_geo(vs), types, s0, cmds, hold, T, record=True)
    d = traj[:, :, :13] - target
    return (d * d).sum(axis=(0, 2)) / d.size  # per-env share of the mean


def _gpu_grads(vs, types, params, s0, cmds, target, hold, T, C=20, mode=0):
    n = len(types)
    sim = Sim(n, types, vs)
    sim.set_adjoint_mode(mode)
    sim.set_params(torch.tensor(params, dtype=torch.float32, device="cuda"))
    coeffs = torch.tensor(params[:, COEF_SLICE], dtype=torch.float32, device="cuda",
                          requires_grad=True)
    acts = torch.tensor(cmds, dtype=torch.float32, device="cuda", requires_grad=True)
    st0 = torch.tensor(s0, dtype=torch.float32, device="cuda")
    traj = rollout(sim, coeffs, acts, st0, hold, T, C)
    tgt = torch.tensor(target, dtype=torch.float32, device="cuda")
    loss = ((traj - tgt) ** 2).mean()
    loss.backward()
    out = (coeffs.grad.double().cpu().numpy(), acts.grad.double().cpu().numpy(),
           traj.detach().double().cpu().numpy())
    sim.close()
    return out


def _rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-30)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("vehicle", [0, 1])
def test_coefficient_gradients_match_fd(vehicle, mode):
    T, hold = 200, 10
    vs, types, params, s0, cmds, target = _problem(T=T, hold=hold, vehicle=vehicle)
    gc, _, traj = _gpu_grads(vs, types, params, s0, cmds, target, hold, T, mode=mode)
    n = len(types)
    fd = np.zeros((n, 18))
    for j in range(18):
        col = COEF_SLICE.start + j
        d = FD_REL * np.abs(params[:, col])
        p1, p2 = params.copy(), params.copy()
        p1[:, col] += d
        p2[:, col] -= d
        fd[:, j] = (_oracle_losses(vs, types, p1, s0, cmds, target, hold, T) -
                    _oracle_losses(vs, types, p2, s0, cmds, target, hold, T)) / (2 * d)
    err = _rel(gc, fd)
    assert err.max() <= TOL_GRAD, (err.max(), np.argmax(err))


@pytest.mark.parametrize("mode", [1, 2])
def test_action_gradients_match_fd(mode):
    T, hold = 200, 10
    vs, types, params, s0, cmds, target = _problem(T=T, hold=hold, seed=3)
    _, ga, _ = _gpu_grads(vs, types, params, s0, cmds, target, hold, T, mode=mode)
    n_seg = cmds.shape[0]
    fd = np.zeros_like(cmds)
    for sg in range(n_seg):
        for i in range(6):
            d = FD_REL * np.maximum(np.abs(cmds[sg, :, i]), 1e-3)
            c1, c2 = cmds.copy(), cmds.copy()
            c1[sg, :, i] += d
            c2[sg, :, i] -= d
            fd[sg, :, i] = (_oracle_losses(vs, types, params, s0, c1, target, hold, T) -
                            _oracle_losses(vs, types, params, s0, c2, target, hold, T)) / (2 * d)
    # per env, all segments and thrusters together
    g = ga.transpose(1, 0, 2).reshape(len(types), -1)
    f = fd.transpose(1, 0, 2).reshape(len(types), -1)
    err = _rel(g, f)
    assert err.max() <= TOL_GRAD, err.max()
    assert np.all(ga[:, :, 6:] == 0)


def test_zero_loss_gradient_gives_zero_and_is_linear():
    T, hold = 60, 10
    vs, types, params, s0, cmds, target = _problem(n=32, T=T, hold=hold, seed=5)
    sim = Sim(32, types, vs)
    sim.set_params(torch.tensor(params, dtype=torch.float32, device="cuda"))
    coeffs = torch.tensor(params[:, COEF_SLICE], dtype=torch.float32, device="cuda",
                          requires_grad=True)
    acts = torch.tensor(cmds, dtype=torch.float32, device="cuda", requires_grad=True)
    st0 = torch.tensor(s0, dtype=torch.float32, device="cuda")
    traj = rollout(sim, coeffs, acts, st0, hold, T, 16)
    g1 = torch.randn_like(traj)
    (gc1, ga1) = torch.autograd.grad(traj, (coeffs, acts), g1, retain_graph=True)
    # scaling by a power of two is exact in FP32, so the adjoint must scale bit for bit
    (gc2, ga2) = torch.autograd.grad(traj, (coeffs, acts), 4.0 * g1, retain_graph=True)
    (gc0, ga0) = torch.autograd.grad(traj, (coeffs, acts), torch.zeros_like(traj))
    assert torch.all(gc0 == 0) and torch.all(ga0 == 0)
    assert torch.equal(gc2, 4.0 * gc1) and torch.equal(ga2, 4.0 * ga1)
    sim.close()


def _general_problem(kind, n=64, T=200, hold=10, seed=11):
    """The FD problem of _problem on the general path: kind "cg" randomises the centre of
    gravity (r_g ~ U[-2, 2] cm per axis), "coupled" adds off-diagonal added mass and linear
    damping at 15 % coupling as well; the target uses the same r_g and extension."""
    vs, types, params, s0, cmds, _ = _problem(n=n, T=T, hold=hold, seed=seed)
    g = np.random.default_rng(200 + seed)
    params[:, I.P_RG:I.P_RG + 3] = I.round_f32(g.uniform(-0.02, 0.02, size=(n, 3)))
    xpar = I.hydro_offdiag(300 + seed, params) if kind == "coupled" else None
    pt = params.copy()
    pt[:, COEF_SLICE] *= np.random.default_rng(99 + seed).uniform(0.9, 1.1, size=(n, 18))
    pt = I.round_f32(pt)
    _, target = O.rollout(pt, oracle_geo(vs), types, s0, cmds, hold, T, record=True, xpar=xpar)
    return vs, types, params, xpar, s0, cmds, I.round_f32(target[:, :, :13])


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("kind", ["cg", "coupled"])
def test_general_path_gradients_match_fd(kind, mode):
    """Off-centre gravity (full M_RB, m r_g coupling in C_RB) and the off-diagonal extension
    (full M_A and D_l): the adjoint's coefficient and action gradients against central finite
    differences of the FP64 oracle, whose mass matrix and terms are built in full."""
    T, hold = 200, 10
    vs, types, params, xpar, s0, cmds, target = _general_problem(kind, T=T, hold=hold)
    n = len(types)
    sim = Sim(n, types, vs)
    sim.set_adjoint_mode(mode)
    sim.set_params(torch.tensor(params, dtype=torch.float32, device="cuda"))
    if xpar is not None:
        sim.set_hydro_offdiag(torch.tensor(xpar, dtype=torch.float32, device="cuda"))
    coeffs = torch.tensor(params[:, COEF_SLICE], dtype=torch.float32, device="cuda",
                          requires_grad=True)
    acts = torch.tensor(cmds, dtype=torch.float32, device="cuda", requires_grad=True)
    st0 = torch.tensor(s0, dtype=torch.float32, device="cuda")
    traj = rollout(sim, coeffs, acts, st0, hold, T, 20)
    tgt = torch.tensor(target, dtype=torch.float32, device="cuda")
    ((traj - tgt) ** 2).mean().backward()
    gc = coeffs.grad.double().cpu().numpy()
    ga = acts.grad.double().cpu().numpy()
    sim.close()

    def losses(p, c):
        _, tr = O.rollout(p, oracle_geo(vs), types, s0, c, hold, T, record=True, xpar=xpar)
        d = tr[:, :, :13] - target
        return (d * d).sum(axis=(0, 2)) / d.size

    fd = np.zeros((n, 18))
    for j in range(18):
        col = COEF_SLICE.start + j
        d = FD_REL * np.abs(params[:, col])
        p1, p2 = params.copy(), params.copy()
        p1[:, col] += d
        p2[:, col] -= d
        fd[:, j] = (losses(p1, cmds) - losses(p2, cmds)) / (2 * d)
    err = _rel(gc, fd)
    assert err.max() <= TOL_GRAD, (kind, err.max(), np.argmax(err))
    # the actions of one segment in the middle of the rollout, every thruster
    sg = cmds.shape[0] // 2
    fa = np.zeros((n, 6))
    for i in range(6):
        d = FD_REL * np.maximum(np.abs(cmds[sg, :, i]), 1e-3)
        c1, c2 = cmds.copy(), cmds.copy()
        c1[sg, :, i] += d
        c2[sg, :, i] -= d
        fa[:, i] = (losses(params, c1) - losses(params, c2)) / (2 * d)
    err = _rel(ga[sg, :, :6], fa)
    assert err.max() <= TOL_GRAD, (kind, err.max())


@pytest.mark.parametrize("n,mixed,T,C,general", [(64, False, 200, 20, False),
                                                 (1000, True, 93, 7, False),
                                                 (4096, False, 50, 32, False),
                                                 (37, True, 5, 1, False),
                                                 (1000, True, 93, 7, True),
                                                 (37, False, 45, 20, True)])
def test_backward_kernels_agree(n, mixed, T, C, general):
    """The two backward kernels (one warp per 32 envs; producer and consumer warps through
    stage records and shared-memory prefetch) evaluate the same per-env operations, every
    multiply-add written as an explicit fmaf, so their coefficient, action and initial-state
    adjoints agree bit for bit: 6-thruster and mixed fleets (8-thruster records), ragged last
    segments and blocks, one-sub-step segments, the diagonal-mass and the general path
    (randomised centre of gravity with the off-diagonal extension)."""
    vs = vehicles()
    types = I.mixed_fleet(3, n, max_group=300) if mixed else np.zeros(n, dtype=np.int32)
    nt = np.array([vs[t].n_thr for t in types])
    hold = 10
    outs = []
    for mode in (1, 2):
        sim = Sim(n, types, vs)
        sim.set_adjoint_mode(mode)
        sim.randomize(77, 0.8, 1.2, 0.2, 0.3, rg_halfwidth=0.02 if general else 0.0)
        if general:
            p = sim.get_params().double().cpu().numpy()
            sim.set_hydro_offdiag(torch.tensor(I.hydro_offdiag(8, p), dtype=torch.float32,
                                               device="cuda"))
        coeffs = sim.get_params()[:, COEF_SLICE].clone().requires_grad_(True)
        acts = torch.tensor(I.commands(5, (T + hold - 1) // hold, n, nt), device="cuda",
                            requires_grad=True)
        s0 = torch.tensor(I.initial_states(21, n), dtype=torch.float32, device="cuda",
                          requires_grad=True)
        traj = rollout(sim, coeffs, acts, s0, hold, T, C)
        g = torch.randn(traj.shape, generator=torch.Generator(device="cuda").manual_seed(3),
                        device="cuda")
        outs.append([x.cpu() for x in torch.autograd.grad(traj, (coeffs, acts, s0), g)])
        sim.close()
    for name, a, b in zip(("coefficients", "actions", "initial state"), *outs):
        torch.testing.assert_close(b, a, rtol=0, atol=0, msg=name)


@pytest.mark.parametrize("general", [False, True])
def test_forward_equals_recorded_steps(general):
    """The rollout's forward runs in one launch (checkpoints written from registers): its
    trajectory, checkpoints and final state equal those of plain recording steps from the same
    start, bit for bit (mixed fleet, ragged last segment; diagonal mass and the general path)."""
    import ctypes
    import math
    from paper_2410_14117_gb300._lib import MG_NSTATE, call
    from paper_2410_14117_gb300.sim import _ptr
    vs = vehicles()
    n, T, C, hold = 1000, 93, 7, 10
    types = I.mixed_fleet(3, n, max_group=300)
    nt = np.array([vs[t].n_thr for t in types])
    acts = torch.tensor(I.commands(5, math.ceil(T / hold), n, nt), device="cuda")
    s0 = torch.tensor(I.initial_states(21, n), dtype=torch.float32, device="cuda")
    sims = []
    for _ in range(2):
        sim = Sim(n, types, vs)
        sim.randomize(77, 0.8, 1.2, 0.2, 0.3, rg_halfwidth=0.02 if general else 0.0)
        if general:
            p = sim.get_params().double().cpu().numpy()
            sim.set_hydro_offdiag(torch.tensor(I.hydro_offdiag(8, p), dtype=torch.float32,
                                               device="cuda"))
        sim.set_state(s0)
        sim.set_actions(acts, hold)
        sims.append(sim)
    a, b = sims
    traj = torch.empty((T, 13, n), device="cuda")
    ckpt = torch.empty((math.ceil(T / C), MG_NSTATE, n), device="cuda")
    step0 = ctypes.c_int64()
    call("mg_rollout_forward", a._h, T, C, _ptr(traj), _ptr(ckpt), ctypes.byref(step0))
    ref = []
    for j in range(math.ceil(T / C)):
        torch.testing.assert_close(ckpt[j].T.contiguous(), b.get_state(), rtol=0, atol=0)
        ref.append(b.step_record(min(C, T - j * C)))
    assert torch.equal(traj, torch.cat(ref))
    assert torch.equal(a.get_state(), b.get_state())
    a.close()
    b.close()
