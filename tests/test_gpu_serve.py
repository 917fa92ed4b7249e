"""Serving pattern: the continuous-batching step server.  Each request's result
is the same alone and in the mix (agents never interact), requests are admitted
by capacity and memory budget, and cancellation / bad requests behave."""
import math
import time

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _hover(p):
    return math.sqrt(p["mass"] * p["g"] / 4.0 / p["k"][2]), 2.0 * p["g"] / p["a_max"] - 1.0


def _request(wl, scene, n, T, seed, u_h, w_h):
    s0 = torch.tensor(np.ascontiguousarray(wl.spawn_states(scene, n, seed, w_h).astype(np.float32).T)).pin_memory()
    u = wl.hover_commands(T, n, seed + 1, u_h).astype(np.float32)
    cm = torch.tensor(np.ascontiguousarray(u.transpose(0, 2, 1))).pin_memory()
    return s0, cm


def _alone(sim, sid, s0, cm, frames):
    """The same request through the plain per-step calls."""
    st = s0.cuda().contiguous()
    n = st.shape[1]
    ids = torch.full((n,), sid, dtype=torch.int32, device="cuda")
    outs = []
    for t in range(cm.shape[0]):
        sim.step(st, cm[t].cuda().contiguous())
        d, c, _ = sim.alloc_images(n)
        sim.render(ids, st, d, c)
        outs.append((d, c))
    torch.cuda.synchronize()
    if frames == "last":
        return st.cpu(), outs[-1][0].cpu(), outs[-1][1].cpu()
    return st.cpu(), torch.stack([o[0] for o in outs]).cpu(), torch.stack([o[1] for o in outs]).cpu()


def _setup(make_sim, wl, budget=0):
    p = wl.params()
    sim = make_sim(p, mem_budget=budget)
    scenes = [wl.room_scene(seed=1), wl.cluttered_scene(n_objects=300, size=(20.0, 20.0, 6.0), seed=3),
              wl.cluttered_scene(n_objects=900, size=(30.0, 30.0, 6.0), seed=4)]
    sids = [sim.add_workload_scene(s) for s in scenes]
    return p, sim, scenes, sids


def _outputs(n, T, frames):
    st = torch.empty((17, n)).pin_memory()
    if frames == "last":
        return st, torch.empty((n, 64, 64)).pin_memory(), torch.empty((n, 64, 64, 3), dtype=torch.uint8).pin_memory()
    return (st, torch.empty((T, n, 64, 64)).pin_memory(),
            torch.empty((T, n, 64, 64, 3), dtype=torch.uint8).pin_memory())


def test_each_request_same_alone_and_in_the_mix(make_sim, wl):
    from paper_2407_14783_b300.serve import Server
    p, sim, scenes, sids = _setup(make_sim, wl)
    w_h, u_h = _hover(p)
    rng = np.random.default_rng(0)
    specs = []
    for k in range(14):
        si = int(rng.integers(0, 3))
        specs.append((si, int(rng.choice([1, 3, 17, 64, 130, 257])), int(rng.integers(1, 7)),
                      "all" if k % 5 == 0 else "last"))
    reqs = []
    with Server(sim, capacity=600) as srv:
        tickets = []
        for k, (si, n, T, fr) in enumerate(specs):
            s0, cm = _request(wl, scenes[si], n, T, 100 + k, u_h, w_h)
            out = _outputs(n, T, fr)
            tickets.append(srv.submit(sids[si], s0, cm, *out, frames=fr))
            reqs.append((si, s0, cm, out, fr))
            if k == 6:
                time.sleep(0.01)      # later arrivals join while earlier ones run
        lat = [srv.wait(t, 60000) for t in tickets]
        st = srv.stats()
    assert all(x > 0 for x in lat)
    assert st["completed"] == len(specs) and st["failed"] == 0
    for si, s0, cm, out, fr in reqs:
        ref = _alone(sim, sids[si], s0, cm, fr)
        for a, b in zip(out, ref):
            assert torch.equal(a, b)


def test_served_requests_match_oracle_sampled(make_sim, oracle_mod, wl):
    """Requests served together (two scenes, 1 to 130 agents, 1 to 5 steps):
    for two sampled agents of each request the final state matches the FP64
    oracle's rollout and the last frame matches the oracle's render of that
    state (depth and colour on unambiguous pixels; misses exact)."""
    from paper_2407_14783_b300.serve import Server
    from parity import DEPTH_TOL, DYN_TOL, dyn_error
    p, sim, scenes, sids = _setup(make_sim, wl)
    w_h, u_h = _hover(p)
    specs = [(1, 1, 3), (2, 130, 5), (1, 64, 1), (2, 17, 4), (0, 3, 2), (2, 100, 2)]
    reqs = []
    with Server(sim, capacity=512) as srv:
        tickets = []
        for k, (si, n, T) in enumerate(specs):
            s0, cm = _request(wl, scenes[si], n, T, 500 + k, u_h, w_h)
            out = _outputs(n, T, "last")
            tickets.append(srv.submit(sids[si], s0, cm, *out, frames="last"))
            reqs.append((si, s0, cm, out))
        for t in tickets:
            srv.wait(t, 60000)
    rng = np.random.default_rng(3)
    for si, s0, cm, (st, depth, rgb) in reqs:
        n = s0.shape[1]
        pick = rng.choice(n, min(2, n), replace=False)
        s0_64 = s0.numpy().T[pick].astype(np.float64)
        u64 = cm.numpy().transpose(0, 2, 1)[:, pick].astype(np.float64)
        ref = oracle_mod.rollout(p, s0_64, u64)[-1]
        got = st.numpy().T[pick]
        assert dyn_error(got, ref)[..., 0:13].max() <= DYN_TOL
        r = oracle_mod.Scene.from_workload(scenes[si]).render(p, got.astype(np.float64))
        d, c = depth.numpy()[pick], rgb.numpy()[pick]
        clear = ~r["tie"]
        assert r["tie"].mean() < 0.01
        assert np.array_equal(c[clear], r["rgb"][clear])
        hitm = clear & (r["id"] >= 0)
        rel = np.abs(d[hitm].astype(np.float64) - r["depth"][hitm]) / r["depth"][hitm]
        assert rel.size == 0 or rel.max() <= DEPTH_TOL
        missm = clear & (r["id"] < 0)
        assert np.all(d[missm] == np.float32(p["max_depth"])) and np.all(c[missm] == 0)


def test_capacity_rejection_and_bad_scene(make_sim, wl):
    from paper_2407_14783_b300.binding import SimError
    from paper_2407_14783_b300.serve import Server
    p, sim, scenes, sids = _setup(make_sim, wl)
    w_h, u_h = _hover(p)
    with Server(sim, capacity=64) as srv:
        s0, cm = _request(wl, scenes[0], 65, 2, 7, u_h, w_h)
        with pytest.raises(SimError):
            srv.submit(sids[0], s0, cm)
        s0, cm = _request(wl, scenes[0], 8, 2, 7, u_h, w_h)
        with pytest.raises(SimError):
            srv.submit(99, s0, cm)
        t = srv.submit(sids[0], s0, cm, *_outputs(8, 2, "last"))
        assert srv.wait(t, 60000) > 0


def test_cancel(make_sim, wl):
    from paper_2407_14783_b300.binding import SimError
    from paper_2407_14783_b300.serve import Server
    p, sim, scenes, sids = _setup(make_sim, wl)
    w_h, u_h = _hover(p)
    with Server(sim, capacity=256) as srv:
        s0, cm = _request(wl, scenes[2], 200, 400, 11, u_h, w_h)
        long_t = srv.submit(sids[2], s0, cm, *_outputs(200, 400, "last"))
        s1, c1 = _request(wl, scenes[1], 100, 3, 12, u_h, w_h)
        queued_t = srv.submit(sids[1], s1, c1, *_outputs(100, 3, "last"))   # waits: 300 > 256 agents
        srv.cancel(queued_t)
        srv.cancel(long_t)
        for t in (queued_t, long_t):
            with pytest.raises(SimError):
                srv.wait(t, 60000)
        s2, c2 = _request(wl, scenes[0], 10, 2, 13, u_h, w_h)
        ok = _outputs(10, 2, "last")
        assert srv.wait(srv.submit(sids[0], s2, c2, *ok), 60000) > 0
        ref = _alone(sim, sids[0], s2, c2, "last")
        assert torch.equal(ok[0], ref[0]) and torch.equal(ok[1], ref[1])
        assert srv.stats()["cancelled"] == 2


def test_memory_admission(make_sim, wl):
    """With a budget that holds the inputs of only a couple of requests at a time,
    later requests wait in the queue and still finish with the right results; a
    request that can never fit fails instead of waiting forever."""
    from paper_2407_14783_b300.binding import SimError
    from paper_2407_14783_b300.serve import Server
    p, sim0, scenes, sids = _setup(make_sim, wl)
    srv0 = Server(sim0, capacity=512)
    w_h, u_h = _hover(p)
    s0, cm = _request(wl, scenes[1], 4, 1, 1, u_h, w_h)
    _alone(sim0, sids[1], s0, cm, "last")      # the context's render-scheduling hints count too
    base = sim0.mem_usage()[0]
    srv0.close()
    n, T = 100, 30
    per_req = 4 * (17 * n + T * 4 * n)
    p, sim, scenes, sids = _setup(make_sim, wl, budget=base + int(2.5 * per_req))
    w_h, u_h = _hover(p)
    # inputs are built first and submitted back to back, so that the budget,
    # not the time between submissions, decides how many wait in the queue
    reqs = []
    for k in range(6):
        s0, cm = _request(wl, scenes[1], n, T, 200 + k, u_h, w_h)
        reqs.append((s0, cm, _outputs(n, T, "last")))
    with Server(sim, capacity=512) as srv:
        tickets = [srv.submit(sids[1], s0, cm, *out) for s0, cm, out in reqs]
        max_queued = 0
        for _ in range(200):
            max_queued = max(max_queued, srv.stats()["queued"])
            if srv.stats()["completed"] == 6:
                break
            time.sleep(0.001)
        for t in tickets:
            srv.wait(t, 60000)
        assert max_queued >= 1
        for s0, cm, out in reqs:
            ref = _alone(sim, sids[1], s0, cm, "last")
            assert torch.equal(out[0], ref[0]) and torch.equal(out[1], ref[1])
        big_s, big_c = _request(wl, scenes[1], 400, 40, 300, u_h, w_h)
        t = srv.submit(sids[1], big_s, big_c, *_outputs(400, 40, "last"))
        with pytest.raises(SimError):
            srv.wait(t, 60000)
