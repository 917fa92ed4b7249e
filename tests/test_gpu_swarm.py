"""Multi-agent (swarm) mode on the GPU against the FP64 oracle: drones of one
scene see each other (Sec. III-B), pairwise proximity, and the mode through
every render path that supports it."""
import numpy as np
import pytest
import torch

from parity import DEPTH_TOL

pytestmark = pytest.mark.gpu

HALF = (0.25, 0.18, 0.06)
RGB = (250, 20, 30)
LABEL = 77


def _cluster(wl, sc, n, seed, spread=1.2):
    """Spawn states pulled into a tight cluster so that the drones see each other."""
    st = wl.spawn_states(sc, n, seed, 1100.0)
    rng = np.random.default_rng(seed)
    centre = st[0, 0:3].copy()
    centre[2] = 2.0
    st[:, 0:3] = centre + rng.uniform(-spread, spread, (n, 3))
    st[:, 2] = np.clip(st[:, 2], 0.6, 3.4)
    return st.astype(np.float32)


def _gpu_render(sim, ids, st, seg=False):
    from paper_2407_14783_b300.sim import to_soa
    n = st.shape[0]
    d, c, h = sim.alloc_images(n, hit=True)
    if seg:
        g = torch.empty_like(h)
        sim.render_seg(ids, to_soa(st), d, c, h, g)
    else:
        sim.render(ids, to_soa(st), d, c, h)
    torch.cuda.synchronize()
    sim.check()
    out = [d.cpu().numpy(), c.cpu().numpy(), h.cpu().numpy()]
    if seg:
        out.append(g.cpu().numpy())
    return out


def _compare(osc, p, st64, ref, d, c, h, id_map=None):
    """Off-tie pixels exact (ids, colour) and within DEPTH_TOL (depth); tie
    pixels admissible for the swarm validator."""
    rid = ref["id"].copy()
    if id_map is not None:
        drone = rid <= -2
        rid[drone] = id_map(rid[drone])
    clear = ~ref["tie"]
    assert np.array_equal(h[clear], rid[clear])
    assert np.array_equal(c[clear], ref["rgb"][clear])
    assert np.all(np.abs(d[clear] - ref["depth"][clear]) <= DEPTH_TOL * ref["depth"][clear])
    ties = np.flatnonzero(ref["tie"].ravel())
    if ties.size:
        hid = h.ravel()[ties]
        if id_map is not None:      # back to the oracle's local drone numbering
            inv = {int(g): int(l) for l, g in id_map.pairs}
            hid = np.array([(-2 - inv[-2 - int(x)]) if x <= -2 else x for x in hid], np.int32)
        ok = osc.validate(p, st64, ties, hid, d.ravel()[ties], swarm={"half": HALF})
        assert ok.all(), f"{(~ok.astype(bool)).sum()} of {ties.size} tie pixels not admissible"
    return int(clear.sum())


@pytest.mark.parametrize("shape", [(8, 4, 1), (16, 2, 1), (8, 8, 2)])
def test_swarm_render_matches_oracle(make_sim, oracle_mod, wl, shape):
    p = wl.params()
    sc = wl.room_scene()
    sim = make_sim(p)
    cfg = sim.render_config()
    cfg.update(tile_w=shape[0], tile_h=shape[1], rays_per_lane=shape[2])
    sim.set_render_config(cfg)
    sid = sim.add_workload_scene(sc)
    sim.set_swarm(HALF, RGB, LABEL)
    n = 24
    st = _cluster(wl, sc, n, 41)
    ids = torch.full((n,), sid, dtype=torch.int32, device="cuda")
    d, c, h = _gpu_render(sim, ids, st)
    osc = oracle_mod.Scene.from_workload(sc)
    ref = osc.render(p, st.astype(np.float64), swarm={"half": HALF, "rgb": RGB})
    assert (ref["id"] <= -2).sum() > 2000          # drones cover a real share of the images
    _compare(osc, p, st.astype(np.float64), ref, d, c, h)


class _Map:
    """Oracle-local drone index -> launch-wide agent index, on id codes."""

    def __init__(self, members):
        self.pairs = list(enumerate(members))
        self.arr = np.asarray(members, np.int32)

    def __call__(self, ids):
        return -2 - self.arr[-2 - ids]


def test_swarm_two_scenes_interleaved(make_sim, oracle_mod, wl):
    """Agents of two scenes interleaved in one launch: each sees only the
    drones of its own scene, reported by their launch-wide index."""
    p = wl.params()
    sa, sb = wl.room_scene(seed=1), wl.room_scene(seed=5)
    sim = make_sim(p)
    ida, idb = sim.add_workload_scene(sa), sim.add_workload_scene(sb)
    sim.set_swarm(HALF, RGB, LABEL)
    n = 30
    sta, stb = _cluster(wl, sa, n // 2, 43), _cluster(wl, sb, n // 2, 44)
    st = np.empty((n, 17), np.float32)
    st[0::2], st[1::2] = sta, stb
    scene = np.array([ida, idb] * (n // 2), np.int32)
    d, c, h = _gpu_render(sim, torch.from_numpy(scene).cuda(), st)
    for sc, members in ((sa, np.arange(0, n, 2)), (sb, np.arange(1, n, 2))):
        osc = oracle_mod.Scene.from_workload(sc)
        sub = st[members].astype(np.float64)
        ref = osc.render(p, sub, swarm={"half": HALF, "rgb": RGB})
        assert (ref["id"] <= -2).sum() > 500
        _compare(osc, p, sub, ref, d[members], c[members], h[members], id_map=_Map(members))


def test_swarm_off_again_and_segmentation(make_sim, oracle_mod, wl):
    p = wl.params()
    sc = wl.room_scene()
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    n = 16
    st = _cluster(wl, sc, n, 45)
    ids = torch.full((n,), sid, dtype=torch.int32, device="cuda")
    plain = _gpu_render(sim, ids, st)
    sim.set_swarm(HALF, RGB, LABEL)
    d, c, h, g = _gpu_render(sim, ids, st, seg=True)
    drone = h <= -2
    assert drone.sum() > 500
    assert np.all(g[drone] == LABEL) and np.all(c[drone] == np.array(RGB, np.uint8))
    assert np.all(d <= plain[0])                    # drones only occlude
    sim.set_swarm(None)
    again = _gpu_render(sim, ids, st)
    for a, b in zip(again, plain):
        assert np.array_equal(a, b)


def test_swarm_env_step_and_loop(make_sim, wl):
    """The streamed host step and the captured loop render the swarm like
    sim_step + sim_render do."""
    from paper_2407_14783_b300.sim import to_soa
    p = wl.params()
    sc = wl.room_scene()
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    sim.set_swarm(HALF, RGB, LABEL)
    n, T = 20, 3
    s0 = to_soa(_cluster(wl, sc, n, 46))
    ids = torch.full((n,), sid, dtype=torch.int32, device="cuda")
    u_hover = 2 * p["g"] / p["a_max"] - 1
    cmds = torch.from_numpy(np.ascontiguousarray(wl.hover_commands(T, n, 47, u_hover, rate_range=0.3)
                                                 .transpose(0, 2, 1))).float()
    # reference: step + render on device buffers
    ref = []
    st = s0.clone()
    for t in range(T):
        sim.step(st, cmds[t].cuda())
        d, c, _ = sim.alloc_images(n)
        sim.render(ids, st, d, c)
        ref.append((d.cpu(), c.cpu()))
    # streamed host step
    st = s0.clone()
    dh = torch.empty((n, 64, 64)).pin_memory()
    ch = torch.empty((n, 64, 64, 3), dtype=torch.uint8).pin_memory()
    for t in range(T):
        sim.env_step(ids, st, cmds[t].contiguous().pin_memory(), dh, ch)
        torch.cuda.synchronize()
        assert torch.equal(dh, ref[t][0]) and torch.equal(ch, ref[t][1])
    # captured loop
    st = s0.clone()
    depth = torch.empty((T, n, 64, 64), device="cuda")
    rgb = torch.empty((T, n, 64, 64, 3), dtype=torch.uint8, device="cuda")
    loop = sim.make_loop(ids, st, cmds.cuda().contiguous(), depth, rgb)
    loop.launch()
    torch.cuda.synchronize()
    sim.check()
    for t in range(T):
        assert torch.equal(depth[t].cpu(), ref[t][0]) and torch.equal(rgb[t].cpu(), ref[t][1])
    loop.close()


def test_swarm_proximity_matches_oracle(make_sim, oracle_mod, wl):
    from paper_2407_14783_b300.sim import to_soa
    p = wl.params()
    sim = make_sim(p)
    sa, sb = sim.add_workload_scene(wl.room_scene(seed=1)), sim.add_workload_scene(wl.room_scene(seed=5))
    rng = np.random.default_rng(48)
    n = 301
    st = np.zeros((n, 17), np.float32)
    st[:, 0:3] = rng.uniform(0.0, 6.0, (n, 3))
    st[:, 6] = 1.0
    scene = rng.integers(0, 2, n).astype(np.int32)
    scene[scene == 0], scene[scene == 1] = sa, sb
    radius = 0.2
    dist, other, hits = sim.swarm_proximity(torch.from_numpy(scene).cuda(), to_soa(st), radius)
    torch.cuda.synchronize()
    sim.check()
    dist, other, hits = dist.cpu().numpy(), other.cpu().numpy(), hits.cpu().numpy()
    pos = st[:, 0:3].astype(np.float64)
    for s in (sa, sb):
        m = np.flatnonzero(scene == s)
        rd, ro, rh = oracle_mod.swarm_proximity(pos[m], radius)
        assert np.allclose(dist[m], rd, rtol=1e-6, atol=1e-6)
        # the nearest agent is unique unless two candidates are within rounding
        d_all = np.linalg.norm(pos[m][:, None] - pos[m][None], axis=2) + np.eye(m.size) * 1e9
        second = np.sort(d_all, axis=1)[:, 1]
        clear = second - rd > 1e-5 * (1 + rd)
        assert np.array_equal(other[m][clear], m[ro[clear]])
        # collision counts, where no pair distance sits on the threshold
        edge = np.any(np.abs(d_all - 2 * radius) < 1e-5, axis=1)
        assert np.array_equal(hits[m][~edge], rh[~edge])
        assert hits[m].sum() > 0


def test_single_agent_swarm_equals_parallel_mode(make_sim, wl):
    """A camera never sees its own drone: one agent per scene renders the same
    in both modes."""
    p = wl.params()
    sa, sb = wl.room_scene(seed=1), wl.room_scene(seed=5)
    sim = make_sim(p)
    ida, idb = sim.add_workload_scene(sa), sim.add_workload_scene(sb)
    st = np.concatenate([_cluster(wl, sa, 1, 50), _cluster(wl, sb, 1, 51)])
    ids = torch.tensor([ida, idb], dtype=torch.int32, device="cuda")
    plain = _gpu_render(sim, ids, st)
    sim.set_swarm(HALF, RGB, LABEL)
    swarm = _gpu_render(sim, ids, st)
    for a, b in zip(plain, swarm):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("n,views", [(600, 6), (4200, 3)])
def test_large_swarm_matches_oracle(make_sim, oracle_mod, wl, n, views):
    """Swarms large enough for the two-level cull (groups of 32 Morton-ordered
    members; beyond 4,096 members per scene the groups keep the bucket order):
    sampled cameras against the oracle rendering the same cameras with the
    whole swarm visible."""
    p = wl.params()
    sc = wl.room_scene()
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    sim.set_swarm(HALF, RGB, LABEL)
    st = wl.spawn_states(sc, n, 60 + n, 1100.0, clearance=0.2).astype(np.float32)
    ids = torch.full((n,), sid, dtype=torch.int32, device="cuda")
    d, c, h = _gpu_render(sim, ids, st)
    pick = np.random.default_rng(n).choice(n, views, replace=False)
    osc = oracle_mod.Scene.from_workload(sc)
    st64 = st.astype(np.float64)
    sw = {"half": HALF, "rgb": RGB, "states": st64, "self": pick}
    ref = osc.render(p, st64[pick], swarm=sw)
    assert (ref["id"] <= -2).sum() > 100 * views       # the other drones fill part of every image
    rid = ref["id"]
    clear = ~ref["tie"]
    assert np.array_equal(h[pick][clear], rid[clear])
    assert np.array_equal(c[pick][clear], ref["rgb"][clear])
    assert np.all(np.abs(d[pick][clear] - ref["depth"][clear]) <= DEPTH_TOL * ref["depth"][clear])
    ties = np.flatnonzero(ref["tie"].ravel())
    if ties.size:
        ok = osc.validate(p, st64[pick], ties, h[pick].ravel()[ties], d[pick].ravel()[ties], swarm=sw)
        assert ok.all(), f"{(~ok).sum()} of {ties.size} tie pixels not admissible"


@pytest.mark.parametrize("wh", [(7, 5), (1, 9), (9, 1), (30, 18)])
def test_large_swarm_ragged_tiles_match_oracle(make_sim, oracle_mod, wl, wh):
    """The larger swarms' frustum cull at image sizes with partial tiles and
    one-pixel-wide or -high images (tile corners clipped to the image; a
    degenerate side plane culls nothing): 600 drones, sampled cameras against
    the oracle."""
    p = wl.params(width=wh[0], height=wh[1])
    sc = wl.room_scene()
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    sim.set_swarm(HALF, RGB, LABEL)
    n = 600
    st = _cluster(wl, sc, n, 90 + wh[0], spread=2.5)
    ids = torch.full((n,), sid, dtype=torch.int32, device="cuda")
    d, c, h = _gpu_render(sim, ids, st)
    pick = np.random.default_rng(wh[0] * 31 + wh[1]).choice(n, 24, replace=False)
    osc = oracle_mod.Scene.from_workload(sc)
    st64 = st.astype(np.float64)
    sw = {"half": HALF, "rgb": RGB, "states": st64, "self": pick}
    ref = osc.render(p, st64[pick], swarm=sw)
    assert (ref["id"] <= -2).any()                     # some sampled pixels see another drone
    clear = ~ref["tie"]
    assert np.array_equal(h[pick][clear], ref["id"][clear])
    assert np.array_equal(c[pick][clear], ref["rgb"][clear])
    assert np.all(np.abs(d[pick][clear] - ref["depth"][clear]) <= DEPTH_TOL * ref["depth"][clear])
    ties = np.flatnonzero(ref["tie"].ravel())
    if ties.size:
        ok = osc.validate(p, st64[pick], ties, h[pick].ravel()[ties], d[pick].ravel()[ties], swarm=sw)
        assert ok.all(), f"{(~ok).sum()} of {ties.size} tie pixels not admissible"
