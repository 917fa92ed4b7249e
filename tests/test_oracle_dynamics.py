"""Pins of the FP64 oracle's dynamics against closed forms and invariants.

Each case reduces the model of Sec. III-A (Eq. 1-4) to a situation with a
textbook solution, so that a dropped term, a wrong sign or a swapped index in
the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest


def _level_state(pos=(1.0, 2.0, 3.0), vel=(0.0, 0.0, 0.0), rates=(0.0, 0.0, 0.0), omega=0.0, yaw=0.0):
    s = np.zeros((1, 17))
    s[0, 0:3] = pos
    s[0, 3:6] = vel
    s[0, 6:10] = [math.cos(yaw / 2), 0.0, 0.0, math.sin(yaw / 2)]
    s[0, 10:13] = rates
    s[0, 13:17] = omega
    return s


def _hover(p):
    w_h = math.sqrt(p["mass"] * p["g"] / 4.0 / p["k"][2])
    u_h = 2.0 * p["g"] / p["a_max"] - 1.0
    return w_h, u_h


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _rotmat(q):
    """Rotation matrix of a unit quaternion via the axis-angle (Rodrigues) form."""
    q = np.asarray(q, float) / np.linalg.norm(q)
    ang = 2.0 * math.atan2(np.linalg.norm(q[1:]), q[0])
    if ang == 0.0:
        return np.eye(3)
    k = q[1:] / np.linalg.norm(q[1:])
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def _same_rotation(qa, qb, tol):
    return min(np.abs(qa - qb).max(), np.abs(qa + qb).max()) < tol


def test_hover_equilibrium(oracle_mod, wl):
    """Level attitude, zero rates, rotors at the hover speed and the hover thrust
    command: the state is a fixed point (any yaw)."""
    p = wl.params()
    w_h, u_h = _hover(p)
    s = _level_state(omega=w_h, yaw=0.7)
    cmds = np.tile(np.array([u_h, 0, 0, 0.0]), (200, 1, 1))
    traj = oracle_mod.rollout(p, s, cmds)
    assert np.abs(traj - s[None]).max() < 1e-9


def test_free_fall_no_thrust(oracle_mod, wl):
    """Rotor speed range [0, 0] gives zero thrust; with Cd = 0 the centre of mass
    falls ballistically whatever the attitude and rates: RK4 integrates the
    quadratic exactly."""
    p = wl.params(omega_min=0.0, omega_max=0.0, Cd=(0.0, 0.0, 0.0))
    s = _level_state(pos=(3.0, -1.0, 20.0), vel=(0.4, -0.3, 1.5), rates=(0.3, -0.2, 0.5))
    T = 150
    rng = np.random.default_rng(0)
    cmds = rng.uniform(-1, 1, (T, 1, 4))
    traj = oracle_mod.rollout(p, s, cmds)
    t = p["dt"] * np.arange(T + 1)
    x_ref = s[0, 0:3] + np.outer(t, s[0, 3:6]) - 0.5 * p["g"] * np.outer(t * t, [0, 0, 1])
    v_ref = s[0, 3:6] + np.outer(t, [0, 0, -p["g"]])
    assert np.abs(traj[:, 0, 0:3] - x_ref).max() < 1e-9
    assert np.abs(traj[:, 0, 3:6] - v_ref).max() < 1e-9
    assert np.abs(traj[:, 0, 13:17]).max() == 0.0


def test_quadratic_drag_closed_form(oracle_mod, wl):
    """No thrust, level and yawed, moving along the body x axis while falling:
    body-frame quadratic drag (Eq. 2, opposing the velocity) gives
    v_x(t) = v0 / (1 + k_x v0 t / m) along the heading and
    v_z(t) = -v_t tanh(g t / v_t), v_t = sqrt(m g / k_z), k = rho Cd s / 2."""
    p = wl.params(omega_min=0.0, omega_max=0.0, Cd=(0.9, 0.7, 1.1), area=(0.05, 0.04, 0.08))
    yaw = 0.6
    v0 = 6.0
    heading = np.array([math.cos(yaw), math.sin(yaw), 0.0])
    s = _level_state(pos=(0, 0, 100.0), vel=v0 * heading, yaw=yaw)
    T = 250
    traj = oracle_mod.rollout(p, s, np.zeros((T, 1, 4)) - 1.0)
    t = p["dt"] * np.arange(T + 1)
    m = p["mass"]
    kx = 0.5 * p["rho"] * p["Cd"][0] * p["area"][0]
    kz = 0.5 * p["rho"] * p["Cd"][2] * p["area"][2]
    vx = v0 / (1.0 + kx * v0 * t / m)
    sx = (m / kx) * np.log1p(kx * v0 * t / m)
    vt = math.sqrt(m * p["g"] / kz)
    vz = -vt * np.tanh(p["g"] * t / vt)
    v = traj[:, 0, 3:6]
    assert np.allclose(v @ heading, vx, rtol=0, atol=1e-7)
    assert np.allclose(v[:, 2], vz, rtol=0, atol=1e-7)
    assert np.allclose((traj[:, 0, 0:3] - s[0, 0:3]) @ heading, sx, rtol=0, atol=1e-7)
    side = np.array([-heading[1], heading[0], 0.0])
    assert np.abs(v @ side).max() < 1e-12


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_rate_loop_first_order_response(oracle_mod, wl, axis):
    """With an instantaneous rotor (c large) and unclamped thrusts, the mixer
    inverse reproduces the desired moment exactly, so a body rate about one
    principal axis follows Omega_n = Omega_d + (Omega_0 - Omega_d)(1 - K h)^n
    (the moment is held over each step, so the rate changes linearly within it)."""
    p = wl.params(c_lag=1e6, Cd=(0.0, 0.0, 0.0))
    w_h, u_h = _hover(p)
    u = np.array([u_h, 0, 0, 0.0])
    u[1 + axis] = 0.3
    rates = [0.0, 0.0, 0.0]
    rates[axis] = -0.4
    s = _level_state(omega=w_h, rates=rates)
    T = 30
    traj = oracle_mod.rollout(p, s, np.tile(u, (T, 1, 1)))
    om_d = 0.3 * p["rate_max"][axis]
    K = p["K_rate"][axis]
    h = p["dt"]
    n = np.arange(T + 1)
    ref = om_d + (-0.4 - om_d) * (1.0 - K * h) ** n
    assert np.abs(traj[:, 0, 10 + axis] - ref).max() < 1e-9
    others = [j for j in range(3) if j != axis]
    assert np.abs(traj[:, 0, 10 + np.array(others)]).max() < 1e-9


def test_rotor_pattern_for_each_rate_axis(oracle_mod, wl):
    """Physical labelling of the X layout (rotor i at 45 + 90 i degrees, spins
    +,-,+,-): a positive roll moment needs more thrust on the +y side (rotors 0
    and 1), a positive pitch moment on the -x side (rotors 1 and 2) and a
    positive yaw moment on the rotors whose reaction torque is +z (0 and 2)."""
    p = wl.params()
    w_h, u_h = _hover(p)
    s = _level_state(omega=w_h)
    for axis, fast in [(0, (0, 1)), (1, (1, 2)), (2, (0, 2))]:
        u = np.array([[u_h, 0, 0, 0.0]])
        u[0, 1 + axis] = 0.2
        out = oracle_mod.step(p, s, u)[0, 13:17]
        slow = [i for i in range(4) if i not in fast]
        assert min(out[list(fast)]) > w_h > max(out[slow]), (axis, out)


def test_collective_thrust_closed_form(oracle_mod, wl):
    """Level, no rates, instantaneous rotors, no drag: u0 maps to a_z = (u0+1)/2 a_max,
    so v_z(t) = (a_z - g) t and z(t) = z0 + (a_z - g) t^2 / 2."""
    p = wl.params(c_lag=1e6, Cd=(0.0, 0.0, 0.0))
    u0 = 0.1
    a = (u0 + 1) / 2 * p["a_max"]
    s = _level_state(pos=(0, 0, 1.0), omega=1000.0)
    T = 50
    traj = oracle_mod.rollout(p, s, np.tile([u0, 0, 0, 0.0], (T, 1, 1)))
    t = p["dt"] * np.arange(1, T + 1)
    assert np.abs(traj[1:, 0, 5] - (a - p["g"]) * t).max() < 1e-9
    assert np.abs(traj[1:, 0, 2] - (1.0 + 0.5 * (a - p["g"]) * t * t)).max() < 1e-9


@pytest.mark.parametrize("n_sub", [1, 4])
def test_rotor_lag_closed_form(oracle_mod, wl, n_sub):
    """Constant desired rotor speed: omega(t) = omega_d + (omega_0 - omega_d) exp(-c t)
    (Eq. 4), independent of the number of physics sub-steps."""
    p = wl.params(n_sub=n_sub)
    w_h, u_h = _hover(p)
    s = _level_state(omega=600.0)
    T = 40
    traj = oracle_mod.rollout(p, s, np.tile([u_h, 0, 0, 0.0], (T, 1, 1)))
    t = p["dt"] * np.arange(T + 1)
    ref = w_h + (600.0 - w_h) * np.exp(-p["c_lag"] * t)
    assert np.abs(traj[:, 0, 13:17] - ref[:, None]).max() < 1e-9 * w_h


def _rotation_case(p, oracle_mod, dt, axis_vec, omega_mag, T_total):
    pp = dict(p, dt=dt)
    q0 = np.array([0.9, 0.1, -0.3, 0.2])
    q0 /= np.linalg.norm(q0)
    s = _level_state(pos=(0, 0, 0))
    s[0, 6:10] = q0
    s[0, 10:13] = omega_mag * np.asarray(axis_vec)
    T = int(round(T_total / dt))
    traj = oracle_mod.rollout(pp, s, np.zeros((T, 1, 4)) - 1.0)
    half = 0.5 * omega_mag * T * dt
    q_ref = _qmul(q0, np.concatenate([[math.cos(half)], math.sin(half) * np.asarray(axis_vec)]))
    q = traj[-1, 0, 6:10]
    return min(np.abs(q - q_ref).max(), np.abs(q + q_ref).max()), traj


def test_constant_rate_rotation_and_rk4_order(oracle_mod, wl):
    """Torque-free spin about a principal axis: q(t) = q0 (x) (cos(|W|t/2), sin(|W|t/2) W/|W|)
    (body-frame rates, Hamilton product).  The global error falls as dt^4 (RK4)."""
    p = wl.params(omega_min=0.0, omega_max=0.0, Cd=(0.0, 0.0, 0.0))
    errs = []
    for dt in (0.08, 0.04, 0.02):
        e, traj = _rotation_case(p, oracle_mod, dt, (0.0, 0.0, 1.0), 3.0, 4.0)
        errs.append(e)
        assert np.abs(traj[:, 0, 10:13] - [0, 0, 3.0]).max() < 1e-12
    assert errs[-1] < 1e-7
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(3.6 < s_ < 4.4 for s_ in slopes), (errs, slopes)


def test_euler_integrator_free_fall(oracle_mod, wl):
    """Explicit Euler on free fall: v_n = v0 - g n h, x_n = x0 + v0 n h - g h^2 n (n-1) / 2."""
    p = wl.params(omega_min=0.0, omega_max=0.0, Cd=(0.0, 0.0, 0.0), integrator=1)
    s = _level_state(pos=(0, 0, 5.0), vel=(1.0, 0.0, 2.0))
    T = 60
    traj = oracle_mod.rollout(p, s, np.zeros((T, 1, 4)) - 1.0)
    n = np.arange(T + 1)
    h = p["dt"]
    assert np.abs(traj[:, 0, 5] - (2.0 - p["g"] * n * h)).max() < 1e-10
    assert np.abs(traj[:, 0, 2] - (5.0 + 2.0 * n * h - p["g"] * h * h * n * (n - 1) / 2)).max() < 1e-10
    assert np.abs(traj[:, 0, 0] - n * h).max() < 1e-10


def test_torque_free_symmetric_top(oracle_mod, wl):
    """J = diag(a, a, c), no moment: Omega_z is constant, (Omega_x, Omega_y) turns at
    lambda = (c - a) Omega_z / a, and the world angular momentum R(q) J Omega and
    the kinetic energy are conserved (pins the gyroscopic term and the frame of
    Omega in the attitude kinematics)."""
    a, c = 0.005, 0.009
    p = wl.params(J=(a, a, c), omega_min=0.0, omega_max=0.0, Cd=(0.0, 0.0, 0.0), dt=0.005)
    s = _level_state()
    s[0, 6:10] = np.array([0.8, 0.2, 0.5, -0.26]) / np.linalg.norm([0.8, 0.2, 0.5, -0.26])
    W0 = np.array([1.2, -0.7, 4.0])
    s[0, 10:13] = W0
    T = 400
    traj = oracle_mod.rollout(p, s, np.zeros((T, 1, 4)) - 1.0)
    t = p["dt"] * np.arange(T + 1)
    lam = (c - a) * W0[2] / a
    z = (W0[0] + 1j * W0[1]) * np.exp(1j * lam * t)
    W = traj[:, 0, 10:13]
    assert np.abs(W[:, 2] - W0[2]).max() < 1e-10
    assert np.abs(W[:, 0] - z.real).max() < 1e-7
    assert np.abs(W[:, 1] - z.imag).max() < 1e-7
    Jd = np.array([a, a, c])
    L0 = _rotmat(traj[0, 0, 6:10]) @ (Jd * W[0])
    E0 = 0.5 * np.sum(Jd * W[0] ** 2)
    for k in range(0, T + 1, 50):
        Lk = _rotmat(traj[k, 0, 6:10]) @ (Jd * W[k])
        assert np.abs(Lk - L0).max() < 1e-8
        assert abs(0.5 * np.sum(Jd * W[k] ** 2) - E0) < 1e-10


def test_quaternion_norm_invariant(oracle_mod, wl):
    """|q| = 1 after every step under random commands."""
    p = wl.params()
    sc = wl.room_scene()
    w_h, _ = _hover(p)
    s = wl.spawn_states(sc, 16, 5, w_h)
    cmds = wl.uniform_commands(100, 16, 6)
    traj = oracle_mod.rollout(p, s, cmds)
    norms = np.linalg.norm(traj[:, :, 6:10], axis=2)
    assert np.abs(norms - 1.0).max() < 1e-12


def test_step_equals_rollout_and_batch_independence(oracle_mod, wl):
    """A rollout is repeated single steps, and agents do not interact (Sec. III-B,
    parallel agents): results do not depend on batch composition."""
    p = wl.params()
    sc = wl.room_scene()
    s = wl.spawn_states(sc, 8, 7, 1100.0)
    cmds = wl.uniform_commands(5, 8, 8)
    traj = oracle_mod.rollout(p, s, cmds)
    y = s
    for t in range(5):
        y = oracle_mod.step(p, y, cmds[t])
        assert np.array_equal(y, traj[t + 1])
    solo = oracle_mod.rollout(p, s[3:4], cmds[:, 3:4])
    assert np.array_equal(solo[:, 0], traj[:, 3])


def test_clamped_thrust_range(oracle_mod, wl):
    """Collective thrust request beyond what the rotors can give (a_max above
    4 f(omega_max) / m): every desired rotor speed clamps at omega_max, so the
    rotors rise as omega_max + (omega_h - omega_max) exp(-c t)."""
    p = wl.params(a_max=80.0)
    w_h = math.sqrt(p["mass"] * p["g"] / 4.0 / p["k"][2])
    s = _level_state(omega=w_h)
    T = 10
    traj = oracle_mod.rollout(p, s, np.tile([1.0, 0, 0, 0], (T, 1, 1)))
    t = p["dt"] * np.arange(T + 1)
    ref = p["omega_max"] + (w_h - p["omega_max"]) * np.exp(-p["c_lag"] * t)
    assert np.abs(traj[:, 0, 13:17] - ref[:, None]).max() < 1e-9 * p["omega_max"]
