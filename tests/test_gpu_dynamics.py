"""GPU dynamics (sim_step, sim_rollout) against the FP64 oracle (Sec. III-A)."""
import math

import numpy as np
import pytest
import torch

from parity import DYN_TOL, dyn_error

pytestmark = pytest.mark.gpu


def _hover(p):
    return math.sqrt(p["mass"] * p["g"] / 4.0 / p["k"][2]), 2.0 * p["g"] / p["a_max"] - 1.0


def _run_gpu_steps(sim, s32, u32):
    from paper_2407_14783_b300.sim import to_soa, from_soa
    st = to_soa(s32)
    out = [from_soa(st)]
    for t in range(u32.shape[0]):
        sim.step(st, to_soa(u32[t]))
        out.append(from_soa(st))
    torch.cuda.synchronize()
    sim.check()
    return np.stack(out)


# Commands for multi-step parity keep every rotor's thrust request away from
# zero (hover thrust, body-rate commands within 30% of the range): near zero
# thrust the square-root inverse of the thrust polynomial has unbounded slope,
# so any last-bit difference of the FP32 state is amplified there.
def _well_conditioned_cmds(wl, steps, n, seed, u_h):
    return wl.hover_commands(steps, n, seed, u_h, rate_range=0.3)


@pytest.mark.parametrize("cmd_kind,steps,tol", [("uniform", 10, DYN_TOL), ("hover", 100, DYN_TOL),
                                                ("uniform", 100, 10 * DYN_TOL)])
def test_step_parity_small(make_sim, oracle_mod, wl, cmd_kind, steps, tol):
    """Tiny configuration: 4 agents in the 492-triangle room; uniform U(-1,1)^4
    commands (10 steps at the stated tolerance; 100 steps, where saturated and
    near-zero rotor thrusts recur, at ten times it) or well-conditioned
    hover-centred commands for 100 steps; FP32 GPU vs FP64 oracle every step."""
    p = wl.params()
    sc = wl.room_scene()
    w_h, u_h = _hover(p)
    n = 4
    s = wl.spawn_states(sc, n, 3, w_h).astype(np.float32)
    u = (wl.uniform_commands(steps, n, 4) if cmd_kind == "uniform" else _well_conditioned_cmds(wl, steps, n, 4, u_h))
    u = u.astype(np.float32)
    ref = oracle_mod.rollout(p, s.astype(np.float64), u.astype(np.float64))
    got = _run_gpu_steps(make_sim(p), s, u)
    err = dyn_error(got, ref)
    body = err[..., 0:13].max()
    assert body <= tol, (cmd_kind, steps, body)
    # rotor speeds: compared in thrust units (the square-root inverse of the thrust
    # polynomial is ill-conditioned near zero thrust, the thrust itself is not)
    k = p["k"]
    f = lambda w: k[2] * w * w + k[1] * w + k[0]
    fmax = f(p["omega_max"])
    rot = np.abs(f(got[..., 13:17]) - f(ref[..., 13:17])).max() / fmax
    assert rot <= DYN_TOL, rot


@pytest.mark.parametrize("n", [1, 31, 129, 1000, 4096])
def test_step_parity_sizes(make_sim, oracle_mod, wl, n):
    """Ragged agent counts across thread blocks; 20 hover-centred steps."""
    p = wl.params()
    sc = wl.cluttered_scene(n_objects=200, size=(20.0, 20.0, 6.0), seed=5)
    w_h, u_h = _hover(p)
    s = wl.spawn_states(sc, n, 7, w_h).astype(np.float32)
    u = _well_conditioned_cmds(wl, 20, n, 8, u_h).astype(np.float32)
    ref = oracle_mod.rollout(p, s.astype(np.float64), u.astype(np.float64))
    got = _run_gpu_steps(make_sim(p), s, u)
    assert dyn_error(got, ref)[..., 0:13].max() <= DYN_TOL


@pytest.mark.parametrize("over", [{"n_sub": 4}, {"integrator": 1}, {"n_sub": 3, "integrator": 1},
                                  {"k": (0.01, 1e-4, 2e-6)}])
def test_step_parity_variants(make_sim, oracle_mod, wl, over):
    """Sub-stepping, the Euler integrator and a full thrust polynomial."""
    p = wl.params(**over)
    sc = wl.room_scene()
    w_h = 1100.0
    u_h = 2.0 * p["g"] / p["a_max"] - 1.0
    s = wl.spawn_states(sc, 64, 9, w_h).astype(np.float32)
    u = _well_conditioned_cmds(wl, 50, 64, 10, u_h).astype(np.float32)
    ref = oracle_mod.rollout(p, s.astype(np.float64), u.astype(np.float64))
    got = _run_gpu_steps(make_sim(p), s, u)
    assert dyn_error(got, ref)[..., 0:13].max() <= DYN_TOL


def test_single_step_parity_uniform_commands(make_sim, oracle_mod, wl):
    """One step of 4096 agents under uniform U(-1,1)^4 commands (clamps active):
    the per-step map agrees with the oracle from identical inputs."""
    p = wl.params()
    sc = wl.cluttered_scene(n_objects=300, size=(20.0, 20.0, 6.0), seed=6)
    w_h, _ = _hover(p)
    n = 4096
    s = wl.spawn_states(sc, n, 13, w_h).astype(np.float32)
    u = wl.uniform_commands(1, n, 14).astype(np.float32)
    ref = oracle_mod.rollout(p, s.astype(np.float64), u.astype(np.float64))
    got = _run_gpu_steps(make_sim(p), s, u)
    assert dyn_error(got, ref)[..., 0:13].max() <= DYN_TOL


def test_rollout_kernel_equals_steps(make_sim, wl):
    """sim_rollout (one launch over T steps) reproduces T sim_step calls bit for bit,
    and its checkpoints are the states at steps 0, K, 2K, ..."""
    from paper_2407_14783_b300.sim import to_soa
    p = wl.params()
    sc = wl.room_scene()
    sim = make_sim(p)
    n, T, K = 300, 23, 5
    s = to_soa(wl.spawn_states(sc, n, 11, 1100.0))
    u = torch.stack([to_soa(x) for x in wl.hover_commands(T, n, 12, -0.6)])
    states, ckpt, final = sim.rollout(s, u, K=K)
    st = s.clone()
    ref = [st.clone()]
    ck = torch.empty_like(st)
    for t in range(T):
        sim.step(st, u[t], ckpt=ck)
        assert torch.equal(ck, ref[-1])
        ref.append(st.clone())
    ref = torch.stack(ref)
    assert torch.equal(states, ref)
    assert torch.equal(final, ref[-1])
    assert torch.equal(ckpt, ref[0:T:K])
    sim.check()


def test_zero_agents_is_a_noop(make_sim, wl):
    sim = make_sim(wl.params())
    st = torch.empty((17, 0), device="cuda")
    sim.step(st, torch.empty((4, 0), device="cuda"))
    sim.check()
