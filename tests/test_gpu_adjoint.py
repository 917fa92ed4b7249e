"""Hand-written adjoint kernels against the oracle's exact (dual number)
derivatives: one step, and a checkpointed rollout through torch.autograd."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from parity import GRAD_RTOL, grad_error


def _hover(p):
    return math.sqrt(p["mass"] * p["g"] / 4.0 / p["k"][2]), 2.0 * p["g"] / p["a_max"] - 1.0


def _check(g, ref, what, tol=GRAD_RTOL):
    """Every component of one agent's gradient within tol of the reference
    (relative, with a floor at GRAD_FLOOR of the agent's largest component)."""
    err, i = grad_error(g, ref)
    assert err < tol, (what, err, i, float(np.ravel(g)[i]), float(np.ravel(ref)[i]))


@pytest.mark.parametrize("over", [{}, {"n_sub": 3}, {"integrator": 1}])
def test_step_backward_matches_oracle_vjp(make_sim, oracle_mod, wl, over):
    from paper_2407_14783_b300.sim import to_soa, from_soa
    p = wl.params(**over)
    w_h, u_h = _hover(p)
    sc = wl.room_scene()
    n = 200
    s = wl.spawn_states(sc, n, 41, w_h).astype(np.float32)
    u = wl.hover_commands(1, n, 42, u_h)[0].astype(np.float32)
    g = np.random.default_rng(4).normal(size=(n, 17)).astype(np.float32)
    ref_s, ref_u = oracle_mod.step_vjp(p, s.astype(np.float64), u.astype(np.float64), g.astype(np.float64))
    sim = make_sim(p)
    gs, gu = sim.step_backward(to_soa(s), to_soa(u), to_soa(g))
    gs, gu = from_soa(gs), from_soa(gu)
    for a in range(n):
        _check(gs[a], ref_s[a], ("state", a))
        _check(gu[a], ref_u[a], ("cmd", a))


def _loss_and_grads(sim, s0, U, goals, lam, K):
    from paper_2407_14783_b300.sim import rollout
    st0 = torch.tensor(s0.T.copy(), device="cuda", requires_grad=True)
    cm = torch.tensor(np.ascontiguousarray(U.transpose(0, 2, 1)), device="cuda", requires_grad=True)
    g = torch.tensor(goals.T.copy(), device="cuda")
    T = U.shape[0]
    states = rollout(sim, st0, cm, K)
    e = states[1:, 0:3, :] - g[None]
    loss = (e * e).sum(dim=(0, 1)) / T + lam * (cm * cm).sum(dim=(0, 1)) / T
    loss.sum().backward()
    return (loss.detach().cpu().numpy(), st0.grad.cpu().numpy().T.astype(np.float64),
            cm.grad.cpu().numpy().transpose(0, 2, 1).astype(np.float64))


@pytest.mark.parametrize("T,K", [(20, 5), (23, 4), (7, 10)])
def test_rollout_gradient_matches_oracle(make_sim, oracle_mod, wl, T, K):
    p = wl.params()
    w_h, u_h = _hover(p)
    sc = wl.room_scene()
    n = 16
    s0 = wl.spawn_states(sc, n, 51, w_h).astype(np.float32)
    U = wl.hover_commands(T, n, 52, u_h).astype(np.float32)
    goals = wl.goal_points(sc, n, 53).astype(np.float32)
    lam = 0.01
    sim = make_sim(p)
    L, gs, gu = _loss_and_grads(sim, s0, U, goals, lam, K)
    Lr, gsr, gur = oracle_mod.rollout_loss_grad(p, s0.astype(np.float64), U.astype(np.float64),
                                                goals.astype(np.float64), lam)
    assert np.allclose(L, Lr, rtol=1e-4)
    for a in range(n):
        full = np.concatenate([gs[a], gu[:, a].ravel()])
        ref = np.concatenate([gsr[a], gur[:, a].ravel()])
        _check(full, ref, a)


@pytest.mark.parametrize("over", [{"integrator": 1}, {"controller": 1}, {"n_sub": 2}])
def test_rollout_gradient_variants_match_oracle(make_sim, oracle_mod, wl, over):
    """The rollout adjoint with the Euler integrator and the SRT controller (both
    through the recorded forward passes) and with two sub-steps per control step
    (re-run forward passes), against the exact FP64 gradient."""
    p = wl.params(**over)
    w_h, u_h = _hover(p)
    sc = wl.room_scene()
    n, T, K = 16, 12, 4
    s0 = wl.spawn_states(sc, n, 81, w_h).astype(np.float32)
    if over.get("controller") == 1:
        u_srt = 2.0 * p["mass"] * p["g"] / 4 / (p["k"][2] * p["omega_max"] ** 2) - 1.0
        U = (u_srt + wl.Rng(82).uniform(-0.02, 0.02, (T, n, 4))).astype(np.float32)
    else:
        U = wl.hover_commands(T, n, 82, u_h).astype(np.float32)
    goals = wl.goal_points(sc, n, 83).astype(np.float32)
    lam = 0.01
    sim = make_sim(p)
    L, gs, gu = _loss_and_grads(sim, s0, U, goals, lam, K)
    Lr, gsr, gur = oracle_mod.rollout_loss_grad(p, s0.astype(np.float64), U.astype(np.float64),
                                                goals.astype(np.float64), lam)
    assert np.allclose(L, Lr, rtol=1e-4)
    for a in range(n):
        full = np.concatenate([gs[a], gu[:, a].ravel()])
        ref = np.concatenate([gsr[a], gur[:, a].ravel()])
        _check(full, ref, a)


def test_rollout_adjoint_tape_grows(make_sim, wl):
    """A context whose tape was sized for a small rollout grows it for a larger
    one (more agents, longer segments) and gives exactly the gradients of a
    fresh context."""
    p = wl.params()
    w_h, u_h = _hover(p)
    sc = wl.room_scene()
    small = make_sim(p)
    s0 = wl.spawn_states(sc, 8, 91, w_h).astype(np.float32)
    U = wl.hover_commands(8, 8, 92, u_h).astype(np.float32)
    goals = wl.goal_points(sc, 8, 93).astype(np.float32)
    _loss_and_grads(small, s0, U, goals, 0.01, 4)
    used = small.mem_usage()[0]
    n, T, K = 48, 24, 8
    s0 = wl.spawn_states(sc, n, 94, w_h).astype(np.float32)
    U = wl.hover_commands(T, n, 95, u_h).astype(np.float32)
    goals = wl.goal_points(sc, n, 96).astype(np.float32)
    L1, gs1, gu1 = _loss_and_grads(small, s0, U, goals, 0.01, K)
    assert small.mem_usage()[0] > used
    L2, gs2, gu2 = _loss_and_grads(make_sim(p), s0, U, goals, 0.01, K)
    assert np.array_equal(L1, L2) and np.array_equal(gs1, gs2) and np.array_equal(gu1, gu2)


def test_rollout_adjoint_without_tape_memory(make_sim, oracle_mod, wl):
    """Under a memory budget too small for the adjoint's tape of forward passes,
    the sweep recomputes them instead: no memory is taken, no error is left
    behind, and the gradients match the taped run's and the FP64 oracle's."""
    p = wl.params()
    w_h, u_h = _hover(p)
    sc = wl.room_scene()
    n, T, K = 32, 20, 5
    s0 = wl.spawn_states(sc, n, 71, w_h).astype(np.float32)
    U = wl.hover_commands(T, n, 72, u_h).astype(np.float32)
    goals = wl.goal_points(sc, n, 73).astype(np.float32)
    lam = 0.01
    taped = make_sim(p)
    L1, gs1, gu1 = _loss_and_grads(taped, s0, U, goals, lam, K)
    probe = make_sim(p)
    base = probe.mem_usage()[0]
    tight = make_sim(p, mem_budget=base + 1024)        # room for nothing more
    L2, gs2, gu2 = _loss_and_grads(tight, s0, U, goals, lam, K)
    assert tight.mem_usage()[0] == base
    assert taped.mem_usage()[0] > base                 # the unconstrained run did keep a tape
    tight.check()
    assert np.allclose(L1, L2, rtol=1e-6)
    Lr, gsr, gur = oracle_mod.rollout_loss_grad(p, s0.astype(np.float64), U.astype(np.float64),
                                                goals.astype(np.float64), lam)
    for a in range(n):
        g1 = np.concatenate([gs1[a], gu1[:, a].ravel()])
        g2 = np.concatenate([gs2[a], gu2[:, a].ravel()])
        ref = np.concatenate([gsr[a], gur[:, a].ravel()])
        # two FP32 evaluations of one gradient that round differently: close as
        # a whole, and each component as close as either is to the exact one
        assert np.linalg.norm(g2 - g1) <= 1e-4 * np.linalg.norm(g1), a
        _check(g2, g1, ("tape-less vs taped", a))
        _check(g2, ref, a)


def test_rollout_gradient_long_horizon_sampled(make_sim, oracle_mod, wl):
    """Differentiable-rollout configuration: 1,024 agents, 200 steps, checkpoints
    every 10 steps; 6 sampled agents checked against the exact FP64 gradient."""
    p = wl.params()
    w_h, u_h = _hover(p)
    sc = wl.cluttered_scene()
    n, T, K = 1024, 200, 10
    s0 = wl.spawn_states(sc, n, 61, w_h).astype(np.float32)
    U = wl.hover_commands(T, n, 62, u_h, rate_range=0.3).astype(np.float32)
    goals = wl.goal_points(sc, n, 63).astype(np.float32)
    lam = 0.01
    sim = make_sim(p)
    L, gs, gu = _loss_and_grads(sim, s0, U, goals, lam, K)
    pick = np.random.default_rng(1).choice(n, 6, replace=False)
    Lr, gsr, gur = oracle_mod.rollout_loss_grad(p, s0[pick].astype(np.float64), U[:, pick].astype(np.float64),
                                                goals[pick].astype(np.float64), lam)
    assert np.allclose(L[pick], Lr, rtol=1e-4)
    for i, a in enumerate(pick):
        full = np.concatenate([gs[a], gu[:, a].ravel()])
        ref = np.concatenate([gsr[i], gur[:, i].ravel()])
        _check(full, ref, a)
