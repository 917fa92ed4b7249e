"""SRT, LV and PS controllers on the GPU against the oracle (Sec. III-A)."""

import numpy as np
import pytest
import torch

from parity import DYN_TOL, dyn_error

pytestmark = pytest.mark.gpu


def _gpu_rollout(sim, s32, u32):
    from paper_2407_14783_b300.sim import to_soa, from_soa
    st = to_soa(s32)
    out = [from_soa(st)]
    for t in range(u32.shape[0]):
        sim.step(st, to_soa(u32[t]))
        out.append(from_soa(st))
    torch.cuda.synchronize()
    sim.check()
    return np.stack(out)


def _yaw(q):
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return np.arctan2(2 * (w * z + x * y), 1 - 2 * (y * y + z * z))


# Commands stay where the controllers are well conditioned: SRT is open loop
# (random per-rotor thrusts make the body tumble, and any last-bit difference
# grows with it), and the geometric attitude error has a saddle at a 180-degree
# yaw error, so yaw targets stay within 1 rad of the current yaw.
def _cmds(wl, ctrl, T, n, spawn, seed):
    rng = wl.Rng(seed)
    if ctrl == 1:
        p = wl.params()
        u_h = 2.0 * p["mass"] * p["g"] / 4 / (p["k"][2] * p["omega_max"] ** 2) - 1.0
        return u_h + rng.uniform(-0.02, 0.02, (T, n, 4))
    tgt = rng.uniform(-1.0, 1.0, (n, 3))
    yaw = (_yaw(spawn[:, 6:10]) + rng.uniform(-1.0, 1.0, n))[:, None]
    if ctrl == 3:
        tgt = spawn[:, 0:3] + 1.5 * tgt
    u = np.concatenate([tgt, yaw], axis=1)
    return np.repeat(u[None], T, axis=0)


@pytest.mark.parametrize("ctrl,steps", [(1, 30), (2, 100), (3, 100)])
def test_controller_parity(make_sim, oracle_mod, wl, ctrl, steps):
    p = wl.params(controller=ctrl)
    sc = wl.room_scene()
    n = 200
    s = wl.spawn_states(sc, n, 70 + ctrl, 1107.0).astype(np.float32)
    u = _cmds(wl, ctrl, steps, n, s, 80 + ctrl).astype(np.float32)
    ref = oracle_mod.rollout(p, s.astype(np.float64), u.astype(np.float64))
    got = _gpu_rollout(make_sim(p), s, u)
    assert dyn_error(got, ref)[..., 0:13].max() <= DYN_TOL


def test_srt_adjoint_and_geometric_backward_refused(make_sim, oracle_mod, wl):
    from paper_2407_14783_b300.binding import SimError
    from paper_2407_14783_b300.sim import to_soa, from_soa
    p = wl.params(controller=1)
    sc = wl.room_scene()
    n = 64
    s = wl.spawn_states(sc, n, 90, 1107.0).astype(np.float32)
    u = _cmds(wl, 1, 1, n, s, 91)[0].astype(np.float32)
    g = np.random.default_rng(9).normal(size=(n, 17)).astype(np.float32)
    ref_s, ref_u = oracle_mod.step_vjp(p, s.astype(np.float64), u.astype(np.float64), g.astype(np.float64))
    sim = make_sim(p)
    gs, gu = sim.step_backward(to_soa(s), to_soa(u), to_soa(g))
    gs, gu = from_soa(gs), from_soa(gu)
    for a in range(n):
        assert np.linalg.norm(gs[a] - ref_s[a]) <= 1e-3 * np.linalg.norm(ref_s[a])
        assert np.linalg.norm(gu[a] - ref_u[a]) <= 1e-3 * max(np.linalg.norm(ref_u[a]), 1e-6)
    lv = make_sim(wl.params(controller=2))
    with pytest.raises(SimError):
        lv.step_backward(to_soa(s), to_soa(u), to_soa(g))


@pytest.mark.parametrize("ctrl", [2, 3])
def test_geometric_rollout_launch(make_sim, oracle_mod, wl, ctrl):
    """sim_rollout with LV / PS (the kernels' geometric instantiation): one launch
    over T steps reproduces T sim_step launches bit for bit, and the oracle
    within the dynamics tolerance."""
    from paper_2407_14783_b300.sim import to_soa, from_soa
    p = wl.params(controller=ctrl)
    sc = wl.room_scene()
    n, T, K = 150, 40, 8
    s = wl.spawn_states(sc, n, 60 + ctrl, 1107.0).astype(np.float32)
    u = _cmds(wl, ctrl, T, n, s, 61 + ctrl).astype(np.float32)
    sim = make_sim(p)
    states, ckpt, final = sim.rollout(to_soa(s), torch.stack([to_soa(x) for x in u]), K=K)
    torch.cuda.synchronize()
    sim.check()
    got = np.stack([from_soa(states[t]) for t in range(T + 1)])
    assert np.array_equal(got, _gpu_rollout(sim, s, u))
    assert np.array_equal(from_soa(final), got[-1])
    ref = oracle_mod.rollout(p, s.astype(np.float64), u.astype(np.float64))
    assert dyn_error(got, ref)[..., 0:13].max() <= DYN_TOL


def test_geometric_yaw_far_from_zero(make_sim, oracle_mod, wl):
    """LV with yaw commands shifted by up to +-60 whole turns: the GPU reduces the
    angle by pi/2 on its own (every quadrant and large quadrant counts), the
    oracle takes FP64 sin and cos of the same float command."""
    p = wl.params(controller=2)
    sc = wl.room_scene()
    n, T = 200, 60
    s = wl.spawn_states(sc, n, 95, 1107.0).astype(np.float32)
    u = _cmds(wl, 2, T, n, s, 96)
    turns = np.random.default_rng(97).integers(-60, 61, n)
    u[:, :, 3] += 2.0 * np.pi * turns[None, :]
    u = u.astype(np.float32)
    ref = oracle_mod.rollout(p, s.astype(np.float64), u.astype(np.float64))
    got = _gpu_rollout(make_sim(p), s, u)
    assert dyn_error(got, ref)[..., 0:13].max() <= DYN_TOL
