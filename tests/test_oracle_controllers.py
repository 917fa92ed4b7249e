"""Pins of the oracle's SRT, LV and PS controllers (Sec. III-A; the paper's
step-response figure is lost, so the pins are closed forms, exact equilibria,
convergence of step responses and invariance under rotations about z)."""
import math

import numpy as np
import pytest


def _state(pos=(0, 0, 2.0), vel=(0, 0, 0), yaw=0.0, rates=(0, 0, 0), omega=0.0):
    s = np.zeros((1, 17))
    s[0, 0:3] = pos
    s[0, 3:6] = vel
    s[0, 6:10] = [math.cos(yaw / 2), 0, 0, math.sin(yaw / 2)]
    s[0, 10:13] = rates
    s[0, 13:17] = omega
    return s


def _yaw(q):
    w, x, y, z = q
    return math.atan2(2 * (w * z + x * y), 1 - 2 * (y * y + z * z))


def _w_hover(p):
    return math.sqrt(p["mass"] * p["g"] / 4 / p["k"][2])


def test_srt_closed_form_and_moment_sign(oracle_mod, wl):
    p = wl.params(controller=1, c_lag=1e6, Cd=(0, 0, 0))
    f_hi = p["k"][2] * p["omega_max"] ** 2
    u = 0.1
    T = 20
    traj = oracle_mod.rollout(p, _state(), np.tile([u, u, u, u], (T, 1, 1)))
    a = 4 * (u + 1) / 2 * f_hi / p["mass"] - p["g"]
    t = p["dt"] * np.arange(T + 1)
    assert np.abs(traj[:, 0, 5] - a * t).max() < 1e-9
    # more thrust on rotors 0 and 1 (the +y side) rolls the body positively
    traj = oracle_mod.rollout(p, _state(), np.tile([0.0, 0.0, -0.2, -0.2], (3, 1, 1)))
    assert traj[-1, 0, 10] > 0 and abs(traj[-1, 0, 11]) < 1e-9


@pytest.mark.parametrize("ctrl", [2, 3])
def test_geometric_equilibrium(oracle_mod, wl, ctrl):
    p = wl.params(controller=ctrl)
    s = _state(pos=(1, 2, 3), yaw=0.7, omega=_w_hover(p))
    u = np.array([[1.0, 2.0, 3.0, 0.7]]) if ctrl == 3 else np.array([[0.0, 0.0, 0.0, 0.7]])
    traj = oracle_mod.rollout(p, s, np.tile(u, (100, 1, 1)))
    assert np.abs(traj - s[None]).max() < 1e-9


def test_lv_step_response_converges(oracle_mod, wl):
    p = wl.params(controller=2)
    s = _state(omega=_w_hover(p))
    vd = np.array([1.0, -0.5, 0.3])
    traj = oracle_mod.rollout(p, s, np.tile(np.r_[vd, 0.4], (200, 1, 1)))
    assert np.abs(traj[-1, 0, 3:6] - vd).max() < 0.02
    assert abs(_yaw(traj[-1, 0, 6:10]) - 0.4) < 0.02


def test_ps_step_response_converges(oracle_mod, wl):
    p = wl.params(controller=3)
    s = _state(pos=(0, 0, 2), omega=_w_hover(p))
    xd = np.array([2.0, -1.0, 2.5])
    traj = oracle_mod.rollout(p, s, np.tile(np.r_[xd, -0.3], (300, 1, 1)))
    assert np.abs(traj[-1, 0, 0:3] - xd).max() < 0.02
    assert np.abs(traj[-1, 0, 3:6]).max() < 0.02
    assert abs(_yaw(traj[-1, 0, 6:10]) + 0.3) < 0.02


@pytest.mark.parametrize("ctrl", [2, 3])
def test_rotation_about_z_equivariance(oracle_mod, wl, ctrl):
    """Rotating the whole problem about world z by th rotates the trajectory."""
    p = wl.params(controller=ctrl)
    th = 0.9
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    s = _state(pos=(1.0, -0.5, 2.0), vel=(0.3, 0.2, -0.1), yaw=0.2, rates=(0.1, -0.2, 0.3), omega=1100.0)
    cmd = np.array([2.0, 1.0, 2.5, 0.5]) if ctrl == 3 else np.array([0.8, -0.4, 0.2, 0.5])
    s_r = s.copy()
    s_r[0, 0:3] = Rz @ s[0, 0:3]
    s_r[0, 3:6] = Rz @ s[0, 3:6]
    qz = np.array([math.cos(th / 2), 0, 0, math.sin(th / 2)])
    w1, x1, y1, z1 = qz
    w2, x2, y2, z2 = s[0, 6:10]
    s_r[0, 6:10] = [w1 * w2 - z1 * z2, w1 * x2 - z1 * y2, w1 * y2 + z1 * x2, w1 * z2 + z1 * w2]
    cmd_r = cmd.copy()
    cmd_r[0:3] = Rz @ cmd[0:3]
    cmd_r[3] = cmd[3] + th
    T = 60
    a = oracle_mod.rollout(p, s, np.tile(cmd, (T, 1, 1)))
    b = oracle_mod.rollout(p, s_r, np.tile(cmd_r, (T, 1, 1)))
    assert np.abs(a[:, 0, 0:3] @ Rz.T - b[:, 0, 0:3]).max() < 1e-9
    assert np.abs(a[:, 0, 10:17] - b[:, 0, 10:17]).max() < 1e-7


@pytest.mark.parametrize("ctrl", [1, 2, 3])
def test_controller_gradients_match_finite_differences(oracle_mod, wl, ctrl):
    p = wl.params(controller=ctrl)
    s = _state(pos=(1.0, -0.5, 2.0), vel=(0.3, 0.2, -0.1), yaw=0.2, rates=(0.1, -0.2, 0.3), omega=1100.0)
    u = (np.array([[0.1, 0.05, -0.05, 0.0]]) if ctrl == 1 else
         np.array([[2.0, 1.0, 2.5, 0.5]]) if ctrl == 3 else np.array([[0.8, -0.4, 0.2, 0.5]]))
    g = np.random.default_rng(ctrl).normal(size=(1, 17))
    gs, gu = oracle_mod.step_vjp(p, s, u, g)
    eps = 1e-6
    for j in range(4):
        up, um = u.copy(), u.copy()
        up[0, j] += eps
        um[0, j] -= eps
        fd = ((oracle_mod.step(p, s, up) - oracle_mod.step(p, s, um)) * g).sum() / (2 * eps)
        assert abs(fd - gu[0, j]) <= 1e-5 * max(1.0, abs(fd)), (j, fd, gu[0, j])
    for j in (0, 4, 7, 11):
        sp, sm = s.copy(), s.copy()
        sp[0, j] += eps
        sm[0, j] -= eps
        fd = ((oracle_mod.step(p, sp, u) - oracle_mod.step(p, sm, u)) * g).sum() / (2 * eps)
        assert abs(fd - gs[0, j]) <= 1e-5 * max(1.0, abs(fd)), (j, fd, gs[0, j])
