"""Pins of the oracle's forward-mode (dual number) derivatives, used to check the
hand-written adjoint of the differentiable dynamics (Sec. III-A)."""
import math

import numpy as np


def _hover(p):
    return math.sqrt(p["mass"] * p["g"] / 4.0 / p["k"][2]), 2.0 * p["g"] / p["a_max"] - 1.0


def test_loss_gradient_free_fall_closed_form(oracle_mod, wl):
    """Zero thrust, no drag: x_t = x0 + v0 t h - g (t h)^2 / 2 z, so for
    L = 1/T sum_t |x_t - g|^2 + lam/T sum_t |u_t|^2 the gradient is
    dL/dx0 = 2/T sum_t (x_t - g), dL/dv0 = 2/T sum_t (x_t - g) t h,
    dL/du_t = 2 lam u_t / T, and zero for attitude, rates and rotor speeds."""
    p = wl.params(omega_min=0.0, omega_max=0.0, Cd=(0.0, 0.0, 0.0))
    T = 25
    h = p["dt"]
    s = np.zeros((1, 17))
    s[0, 0:3] = [1.0, -2.0, 8.0]
    s[0, 3:6] = [0.3, 0.2, 1.0]
    s[0, 6:10] = np.array([0.9, 0.1, 0.2, -0.1]) / np.linalg.norm([0.9, 0.1, 0.2, -0.1])
    s[0, 10:13] = [0.2, -0.1, 0.4]
    rng = np.random.default_rng(1)
    U = rng.uniform(-0.9, 0.9, (T, 1, 4))
    goal = np.array([[2.0, 1.0, 3.0]])
    lam = 0.01
    loss, gs, gc = oracle_mod.rollout_loss_grad(p, s, U, goal, lam)
    t = h * np.arange(1, T + 1)
    x = s[0, 0:3] + np.outer(t, s[0, 3:6]) - 0.5 * p["g"] * np.outer(t * t, [0, 0, 1])
    e = x - goal[0]
    L_ref = (e * e).sum() / T + lam * (U * U).sum() / T
    assert abs(loss[0] - L_ref) < 1e-10
    assert np.abs(gs[0, 0:3] - 2.0 / T * e.sum(0)).max() < 1e-9
    assert np.abs(gs[0, 3:6] - 2.0 / T * (e * t[:, None]).sum(0)).max() < 1e-9
    assert np.abs(gs[0, 6:17]).max() < 1e-12
    assert np.abs(gc - 2 * lam * U / T).max() < 1e-12


def test_loss_gradient_matches_central_differences(oracle_mod, wl):
    """Exact derivatives agree with central differences (h = 1e-3) of the loss
    computed from the oracle's own trajectories, on hover-centred rollouts."""
    p = wl.params()
    scn = wl.room_scene()
    w_h, u_h = _hover(p)
    n, T = 2, 12
    s0 = wl.spawn_states(scn, n, 21, w_h)
    U = wl.hover_commands(T, n, 22, u_h)
    goals = wl.goal_points(scn, n, 23)
    lam = 0.01
    loss, gs, gc = oracle_mod.rollout_loss_grad(p, s0, U, goals, lam)
    traj = oracle_mod.rollout(p, s0, U)
    assert np.allclose(loss, oracle_mod.rollout_loss(traj, U, goals, lam), rtol=1e-13, atol=0)
    eps = 1e-3
    rng = np.random.default_rng(2)
    for a in range(n):
        def L(s_a, U_a):
            s = s0.copy(); s[a] = s_a
            u = U.copy(); u[:, a] = U_a
            return oracle_mod.rollout_loss(oracle_mod.rollout(p, s, u), u, goals, lam)[a]
        for j in list(range(17)):
            sp, sm = s0[a].copy(), s0[a].copy()
            sp[j] += eps; sm[j] -= eps
            fd = (L(sp, U[:, a]) - L(sm, U[:, a])) / (2 * eps)
            assert abs(fd - gs[a, j]) <= 1e-4 * max(1.0, abs(gs[a, j])), (a, j, fd, gs[a, j])
        for k in rng.choice(T * 4, 12, replace=False):
            t, j = divmod(int(k), 4)
            Up, Um = U[:, a].copy(), U[:, a].copy()
            Up[t, j] += eps; Um[t, j] -= eps
            fd = (L(s0[a], Up) - L(s0[a], Um)) / (2 * eps)
            assert abs(fd - gc[t, a, j]) <= 1e-4 * max(1.0, abs(gc[t, a, j])), (a, t, j, fd, gc[t, a, j])


def test_step_vjp_matches_central_differences(oracle_mod, wl):
    """One-step vector-Jacobian product against central differences."""
    p = wl.params()
    scn = wl.room_scene()
    w_h, u_h = _hover(p)
    s = wl.spawn_states(scn, 3, 31, w_h)
    u = wl.hover_commands(1, 3, 32, u_h)[0]
    rng = np.random.default_rng(3)
    g = rng.normal(size=(3, 17))
    gs, gc = oracle_mod.step_vjp(p, s, u, g)
    # small step: rotor speeds near the steep part of the thrust inverse make the
    # O(eps^2) truncation term visible in the weighted sum at eps = 1e-4
    eps = 1e-6
    for j in range(17):
        sp, sm = s.copy(), s.copy()
        sp[:, j] += eps; sm[:, j] -= eps
        fd = ((oracle_mod.step(p, sp, u) - oracle_mod.step(p, sm, u)) * g).sum(1) / (2 * eps)
        assert np.allclose(fd, gs[:, j], rtol=1e-6, atol=1e-5), (j, fd, gs[:, j])
    for j in range(4):
        up, um = u.copy(), u.copy()
        up[:, j] += eps; um[:, j] -= eps
        fd = ((oracle_mod.step(p, s, up) - oracle_mod.step(p, s, um)) * g).sum(1) / (2 * eps)
        assert np.allclose(fd, gc[:, j], rtol=1e-6, atol=1e-5), (j, fd, gc[:, j])
