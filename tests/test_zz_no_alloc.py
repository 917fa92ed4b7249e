"""The allocation-free render entry point, sim_render_scene_static.

Callers that cannot allocate device memory while they run (a control loop that
must not touch the allocator after set-up, a process whose device memory all
belongs to another framework's pool) use this entry point instead of
sim_render_scene, which allocates an agent -> scene id array on every call.
It must give the same images, call after call, although every call reuses one
static device array.  This file is collected last on purpose.
"""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


def _call(L, fn, sim, n, sid, state, d, c, h):
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    return getattr(L, fn)(sim.h, n, sid, p(state), p(d), p(c), p(h), s)


def test_static_render_matches_render_scene_twice(make_sim, wl):
    from paper_2407_14783_b300 import binding
    from paper_2407_14783_b300.sim import to_soa
    L = binding.lib()
    p = wl.params()
    sim = make_sim(p)
    scenes = [wl.room_scene(seed=1), wl.cluttered_scene(n_objects=300, size=(20.0, 20.0, 6.0), seed=8)]
    sids = [sim.add_workload_scene(sc) for sc in scenes]
    # two calls in a row with different scenes and agent counts: the shared id
    # array is refilled and the counters cleared each time
    for sid, sc, n, seed in [(sids[1], scenes[1], 97, 21), (sids[0], scenes[0], 13, 22)]:
        st = to_soa(wl.spawn_states(sc, n, seed, 1100.0))
        d0, c0, h0 = sim.alloc_images(n, hit=True)
        d1, c1, h1 = sim.alloc_images(n, hit=True)
        assert _call(L, "sim_render_scene", sim, n, sid, st, d0, c0, h0) == 0
        assert _call(L, "sim_render_scene_static", sim, n, sid, st, d1, c1, h1) == 0
        torch.cuda.synchronize()
        sim.check()
        assert torch.equal(h1, h0) and torch.equal(c1, c0)
        rel = ((d1 - d0).abs() / d0).max().item()
        assert rel <= 1e-4
        assert (h0 >= 0).float().mean().item() > 0.5


def test_static_render_rejects_too_many_agents(make_sim, wl):
    from paper_2407_14783_b300 import binding
    L = binding.lib()
    sim = make_sim(wl.params())
    sid = sim.add_workload_scene(wl.room_scene())
    n = 65537
    st = torch.zeros((17, 1), device="cuda")
    d = torch.zeros((1,), device="cuda")
    rc = _call(L, "sim_render_scene_static", sim, n, sid, st, d, d, d)
    assert rc == -1   # SIM_ERR_INVALID_ARG, nothing launched
    assert b"SIM_RENDER_STATIC_MAX_AGENTS" in L.sim_last_error(sim.h)
