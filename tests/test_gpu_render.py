"""GPU LBVH build + persistent ray cast against the FP64 oracle (Sec. III-B)."""
import numpy as np
import pytest
import torch

from parity import compare_images

pytestmark = pytest.mark.gpu


def _render(sim, sid_or_ids, s32):
    from paper_2407_14783_b300.sim import to_soa
    n = s32.shape[0]
    st = to_soa(s32)
    ids = sid_or_ids if isinstance(sid_or_ids, torch.Tensor) else torch.full((n,), sid_or_ids, dtype=torch.int32,
                                                                             device="cuda")
    d, c, h = sim.alloc_images(n, hit=True)
    sim.render(ids, st, d, c, h)
    torch.cuda.synchronize()
    sim.check()
    return d.cpu().numpy(), c.cpu().numpy(), h.cpu().numpy()


def test_render_parity_tiny(make_sim, oracle_mod, wl):
    """492-triangle room, 4 agents (the tiny configuration)."""
    p = wl.params()
    sc = wl.room_scene()
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    s = wl.spawn_states(sc, 4, 3, 1100.0).astype(np.float32)
    d, c, h = _render(sim, sid, s)
    stats = compare_images(oracle_mod.Scene.from_workload(sc), p, s.astype(np.float64), d, c, h)
    assert stats["hit_frac"] > 0.9


def test_render_parity_large_scene_sampled(make_sim, oracle_mod, wl):
    """208,812-triangle cluttered room at the benchmark's launch shape (256 agents,
    one launch); the oracle checks 24 sampled agents' full images."""
    p = wl.params()
    sc = wl.cluttered_scene()
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    info = sim.scene_info(sid)
    assert info["n_tris"] == sc.n_tris and info["n_large"] == 12
    s = wl.spawn_states(sc, 256, 3, 1100.0).astype(np.float32)
    d, c, h = _render(sim, sid, s)
    pick = np.random.default_rng(0).choice(256, 24, replace=False)
    compare_images(oracle_mod.Scene.from_workload(sc), p, s[pick].astype(np.float64), d[pick], c[pick], h[pick])


def test_render_configs_identical(make_sim, wl):
    """Every supported tile shape / rays-per-lane / stack placement and depth /
    node width gives the same images (the closest-hit rule with lowest-id ties
    is order independent); a binary stack shallower than the scene's BVH is
    refused."""
    from paper_2407_14783_b300.binding import SimError
    from paper_2407_14783_b300.sim import Sim
    p = wl.params()
    sc = wl.cluttered_scene(n_objects=400, size=(20.0, 20.0, 6.0), seed=4)
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    depth = sim.scene_info(sid)["depth"]
    assert 0 < depth < 32
    s = wl.spawn_states(sc, 37, 5, 1100.0).astype(np.float32)
    cfgs = Sim.render_configs()
    assert {c["stack_depth"] for c in cfgs} == {32, 48, 64}
    base = None
    for cfg in cfgs:
        sim.set_render_config(cfg)
        out = _render(sim, sid, s)
        if base is None:
            base = out
        else:
            for a, b in zip(out, base):
                assert np.array_equal(a, b), cfg
    # a 2M-triangle scene's tree is deeper than 32 levels: 32-entry stacks are refused
    big = sim.add_workload_scene(wl.sized_scene(2_000_000, 711))
    if sim.scene_info(big)["depth"] > 32:
        sim.set_render_config({**cfgs[0], "stack_depth": 32, "stack_in_smem": 0, "node_width": 2})
        with pytest.raises(SimError):
            _render(sim, sid, s)


def test_stack_as_deep_as_tree(make_sim, oracle_mod, wl):
    """A binary walk holds at most one stack entry per internal node of its root
    path, so a stack of exactly the tree's depth suffices: the 208,812-triangle
    scene (a PLOC tree 32 levels deep) renders with 32-entry stacks, in
    registers and in shared memory, exactly as with 64-entry ones, without a
    traversal error, and matches the oracle."""
    from paper_2407_14783_b300.sim import Sim
    p = wl.params()
    sc = wl.cluttered_scene(seed=2)
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    depth = sim.scene_info(sid)["depth"]
    assert 24 <= depth <= 32
    s = wl.spawn_states(sc, 128, 17, 1100.0).astype(np.float32)
    cfgs = [c for c in Sim.render_configs() if c["node_width"] == 2 and c["tile_w"] == 8 and c["tile_h"] == 4
            and c["stage_in_smem"] == 0]
    ref = None
    for cfg in sorted(cfgs, key=lambda c: -c["stack_depth"]):
        sim.set_render_config(cfg)
        out = _render(sim, sid, s)
        if ref is None:
            ref = out
            pick = np.random.default_rng(5).choice(128, 6, replace=False)
            compare_images(oracle_mod.Scene.from_workload(sc), p, s[pick].astype(np.float64), out[0][pick],
                           out[1][pick], out[2][pick])
        else:
            for a, b in zip(out, ref):
                assert np.array_equal(a, b), cfg
    assert {c["stack_depth"] for c in cfgs} >= {32, 64}


@pytest.mark.parametrize("wh", [(30, 18), (64, 64), (128, 96), (7, 5)])
def test_render_ragged_image_sizes(make_sim, oracle_mod, wl, wh):
    """Image sizes that leave partial tiles."""
    p = wl.params(width=wh[0], height=wh[1])
    sc = wl.room_scene()
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    s = wl.spawn_states(sc, 5, 6, 1100.0).astype(np.float32)
    d, c, h = _render(sim, sid, s)
    compare_images(oracle_mod.Scene.from_workload(sc), p, s.astype(np.float64), d, c, h, max_tie_frac=0.02)


def test_multi_scene_one_launch_equals_per_scene(make_sim, oracle_mod, wl):
    """Scenes of uneven size in one launch through the scene table give the same
    images as rendering each scene's agents alone, and match the oracle."""
    p = wl.params()
    scenes = [wl.room_scene(seed=1), wl.cluttered_scene(n_objects=50, size=(10.0, 10.0, 4.0), seed=2),
              wl.cluttered_scene(n_objects=600, size=(25.0, 25.0, 6.0), seed=3)]
    sim = make_sim(p)
    sids = [sim.add_workload_scene(s) for s in scenes]
    counts = [3, 9, 20]
    states = [wl.spawn_states(s, k, 10 + i, 1100.0).astype(np.float32) for i, (s, k) in enumerate(zip(scenes, counts))]
    all_s = np.concatenate(states)
    ids = torch.tensor(np.repeat(sids, counts), dtype=torch.int32, device="cuda")
    d, c, h = _render(sim, ids, all_s)
    off = 0
    for sc, sid, st, k in zip(scenes, sids, states, counts):
        d1, c1, h1 = _render(sim, sid, st)
        assert np.array_equal(d[off:off + k], d1) and np.array_equal(c[off:off + k], c1)
        assert np.array_equal(h[off:off + k], h1)
        compare_images(oracle_mod.Scene.from_workload(sc), p, st.astype(np.float64), d1, c1, h1)
        off += k


def test_degenerate_scenes(make_sim, oracle_mod, wl):
    """Empty scene (all misses), a single triangle, and a scene of only large
    triangles (no BVH)."""
    p = wl.params()
    sim = make_sim(p)
    s = np.zeros((2, 17), np.float32)
    s[:, 6] = 1.0
    s[1, 0:3] = [0.5, 0.2, -0.1]
    e = sim.add_scene(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 3)))
    d, c, h = _render(sim, e, s)
    assert np.all(h == -1) and np.all(d == p["max_depth"]) and np.all(c == 0)
    v = np.array([[3.0, -1.0, -1.0], [3.0, 1.5, -1.0], [3.0, 0.0, 2.0]])
    one = sim.add_scene(v, [[0, 1, 2]], [[10, 20, 30]])
    d, c, h = _render(sim, one, s)
    compare_images(oracle_mod.Scene(v, [[0, 1, 2]], [[10, 20, 30]]), p, s.astype(np.float64), d, c, h,
                   max_tie_frac=0.05)
    bv, bf = wl.box_mesh((-5, -5, -3), (5, 5, 3))
    rgb = np.arange(36, dtype=np.uint8).reshape(12, 3)
    big = sim.add_scene(bv, bf, rgb)
    assert sim.scene_info(big)["n_large"] == 12
    d, c, h = _render(sim, big, s)
    compare_images(oracle_mod.Scene(bv, bf, rgb), p, s.astype(np.float64), d, c, h, max_tie_frac=0.05)


def test_unknown_scene_is_reported(make_sim, wl):
    p = wl.params()
    sim = make_sim(p)
    sid = sim.add_workload_scene(wl.room_scene())
    s = np.zeros((3, 17), np.float32)
    s[:, 6] = 1.0
    s[:, 0:3] = (5.0, 5.0, 2.0)     # inside the 10 x 10 x 4 m room
    ids = torch.tensor([sid, 7, sid], dtype=torch.int32, device="cuda")
    from paper_2407_14783_b300.sim import to_soa
    d, c, h = sim.alloc_images(3, hit=True)
    sim.render(ids, to_soa(s), d, c, h)
    assert sim.status() == -4          # SIM_ERR_NOT_FOUND, read and cleared
    assert sim.status() == 0
    assert torch.all(h[1] == -1) and torch.all(h[0] >= 0)


def test_scheduling_hints_do_not_change_images(make_sim, wl):
    """Renders after the first reorder work from the previous launch's tile costs;
    images must equal a fresh context's, also when the agent count changes."""
    from paper_2407_14783_b300.sim import to_soa
    p = wl.params()
    sc = wl.cluttered_scene(n_objects=800, size=(25.0, 25.0, 6.0), seed=9)
    a = make_sim(p)
    sa = a.add_workload_scene(sc)
    s = wl.spawn_states(sc, 96, 17, 1100.0).astype(np.float32)
    outs = [_render(a, sa, s) for _ in range(4)]          # launches 2.. use hints
    small = _render(a, sa, s[:40])                          # different item count
    again = _render(a, sa, s)
    b = make_sim(p)
    sb = b.add_workload_scene(sc)
    fresh = _render(b, sb, s)
    fresh_small = _render(b, sb, s[:40])
    for o in outs + [again]:
        for x, y in zip(o, fresh):
            assert np.array_equal(x, y)
    for x, y in zip(small, fresh_small):
        assert np.array_equal(x, y)


def test_render_maximum_image_size(make_sim, oracle_mod, wl):
    """The largest image the library accepts (1024 x 1024) on the large scene:
    two agents, every pixel against the oracle."""
    p = wl.params(width=1024, height=1024)
    sc = wl.cluttered_scene()
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    s = wl.spawn_states(sc, 2, 17, 1100.0).astype(np.float32)
    d, c, h = _render(sim, sid, s)
    compare_images(oracle_mod.Scene.from_workload(sc), p, s.astype(np.float64), d, c, h, max_tie_frac=0.02)
    with pytest.raises(Exception):
        make_sim(wl.params(width=1025, height=64))


def test_bounded_status_wait_times_out_then_succeeds(make_sim, wl):
    """sim_get_status gives up after its deadline while the stream is still busy
    (SIM_ERR_TIMEOUT, nothing faults or hangs), and succeeds once it drains."""
    from paper_2407_14783_b300.sim import to_soa
    p = wl.params()
    sc = wl.cluttered_scene()
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    n = 4096
    st = to_soa(wl.spawn_states(sc, n, 21, 1100.0).astype(np.float32))
    ids = torch.full((n,), sid, dtype=torch.int32, device="cuda")
    d, c, _ = sim.alloc_images(n)
    torch.cuda.synchronize()
    for _ in range(4):
        sim.render(ids, st, d, c)            # a few milliseconds of queued work
    rc = sim.status(timeout_ms=0)
    assert rc == -6                           # SIM_ERR_TIMEOUT
    assert sim.status(timeout_ms=60000) == 0
    assert torch.isfinite(d).all()


def test_outputs_finite_and_in_range(make_sim, wl):
    """No NaN or Inf anywhere: depth in (0, max_depth], hit ids in range, and
    the state after 100 steps of uniform commands."""
    from paper_2407_14783_b300.sim import to_soa
    p = wl.params()
    sc = wl.cluttered_scene()
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    n = 128
    st = to_soa(wl.spawn_states(sc, n, 22, 1100.0).astype(np.float32))
    cm = torch.from_numpy(np.ascontiguousarray(wl.uniform_commands(100, n, 23).transpose(0, 2, 1))).float().cuda()
    for t in range(100):
        sim.step(st, cm[t])
    ids = torch.full((n,), sid, dtype=torch.int32, device="cuda")
    d, c, h = sim.alloc_images(n, hit=True)
    sim.render(ids, st, d, c, h)
    torch.cuda.synchronize()
    sim.check()
    assert torch.isfinite(st).all()
    assert torch.isfinite(d).all() and (d > 0).all() and (d <= p["max_depth"]).all()
    assert ((h >= -1) & (h < sc.n_tris)).all()


def test_tile_costs_and_build_times(make_sim, wl):
    """The load-analysis queries: per-tile traversal costs of the last render
    (refused before any render) and the phase times of a scene's build."""
    from paper_2407_14783_b300.binding import SimError
    p = wl.params()
    sc = wl.cluttered_scene(n_objects=400, size=(20.0, 20.0, 6.0), seed=4)
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    with pytest.raises(SimError):
        sim.tile_costs()
    bt = sim.scene_build_times(sid)
    assert set(bt) == set(sim.BUILD_PHASES) | {"wall"}
    assert all(v >= 0.0 for v in bt.values()) and bt["clustering"] > 0.0 and bt["sort"] > 0.0
    assert bt["wall"] >= max(bt[k] for k in sim.BUILD_PHASES)
    n = 9
    s = wl.spawn_states(sc, n, 5, 1100.0).astype(np.float32)
    _render(sim, sid, s)
    cfg = sim.render_config()
    costs = sim.tile_costs()
    assert costs.shape == (n, -(-64 // cfg["tile_h"]), -(-64 // cfg["tile_w"]))
    assert (costs >= 1).all()            # every tile walks at least the root
    assert costs.max() > 4 * np.median(costs)   # and the costs are uneven, which is why they are scheduled


def test_kernel_timing(make_sim, wl):
    """sim_kernel_timing: every ray-cast launch while timing is on records its
    kernel time (positive, below the whole render's), the images are those of
    an untimed launch, and reading or disabling clears the record."""
    p = wl.params()
    sc = wl.room_scene()
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    s = wl.spawn_states(sc, 64, 8, 1100.0).astype(np.float32)
    base = _render(sim, sid, s)
    sim.kernel_timing(True)
    outs = [_render(sim, sid, s) for _ in range(3)]
    ms = sim.kernel_times()
    assert len(ms) == 3 and np.all(ms > 0) and np.all(ms < 1000)
    for out in outs:
        for a, b in zip(out, base):
            assert np.array_equal(a, b)
    assert len(sim.kernel_times()) == 0
    _render(sim, sid, s)
    sim.kernel_timing(False)
    _render(sim, sid, s)
    assert len(sim.kernel_times()) == 0
    # launches captured into a graph (a step loop) record no events, and the
    # loop's replays record none either; eager launches after it still do
    from paper_2407_14783_b300.sim import to_soa
    n = s.shape[0]
    ids = torch.full((n,), sid, dtype=torch.int32, device="cuda")
    st = to_soa(s)
    cmds = torch.zeros((3, 4, n), dtype=torch.float32, device="cuda")
    d = torch.zeros((2, n, p["height"], p["width"]), dtype=torch.float32, device="cuda")
    sim.kernel_timing(True)
    loop = sim.make_loop(ids, st, cmds, d)
    loop.launch()
    torch.cuda.synchronize()
    assert len(sim.kernel_times()) == 0
    _render(sim, sid, s)
    assert len(sim.kernel_times()) == 1
    loop.close()
    sim.kernel_timing(False)
