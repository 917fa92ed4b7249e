"""Nearest-obstacle query on the GPU against the FP64 brute-force oracle."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _tol(d):
    return 5e-5 + 1e-5 * d


def _check(sim, osc, ids, s32, max_dist):
    from paper_2407_14783_b300.sim import to_soa
    d, q, t = sim.nearest_obstacle(ids, to_soa(s32), max_dist)
    torch.cuda.synchronize()
    sim.check()
    d, q, t = d.cpu().numpy(), q.cpu().numpy().T, t.cpu().numpy()
    pos = s32[:, 0:3].astype(np.float64)
    dr, qr, tr = osc.nearest(pos, max_dist)
    assert np.all(np.abs(d - dr) <= _tol(dr)), np.abs(d - dr).max()
    hit = tr >= 0
    assert np.array_equal(t >= 0, hit)
    # the reported triangle is (one of) the nearest, and the point lies at the distance
    dt = osc.point_triangle(pos[hit], t[hit])
    assert np.all(np.abs(dt - dr[hit]) <= _tol(dr[hit]))
    assert np.all(np.abs(np.linalg.norm(q[hit] - pos[hit], axis=1) - d[hit]) <= _tol(d[hit]))
    assert np.all(d[~hit] == np.float32(max_dist)) and np.array_equal(q[~hit], s32[~hit, 0:3])
    return d


def test_nearest_large_scene(make_sim, oracle_mod, wl):
    p = wl.params()
    sc = wl.cluttered_scene()
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    s = wl.spawn_states(sc, 256, 3, 1100.0).astype(np.float32)
    ids = torch.full((256,), sid, dtype=torch.int32, device="cuda")
    osc = oracle_mod.Scene.from_workload(sc, bvh=False)
    d = _check(sim, osc, ids, s, 100.0)
    assert d.min() >= 0.3 - 1e-4        # spawns keep 0.3 m clearance
    _check(sim, osc, ids, s, 0.6)        # some agents have nothing within 0.6 m


def test_nearest_multi_scene_and_walls_only(make_sim, oracle_mod, wl):
    p = wl.params()
    scenes = [wl.room_scene(seed=1), wl.cluttered_scene(n_objects=150, size=(15.0, 15.0, 5.0), seed=6)]
    bv, bf = wl.box_mesh((0, 0, 0), (8, 7, 3))
    scenes.append(wl.Scene(bv.astype(np.float32), bf.astype(np.int32), np.zeros((12, 3), np.uint8),
                           (np.zeros(3), np.array([8, 7, 3.0])), np.zeros((0, 2, 3))))
    sim = make_sim(p)
    sids = [sim.add_workload_scene(s) for s in scenes]
    for sid, sc, k in zip(sids, scenes, (7, 33, 5)):
        s = wl.spawn_states(sc, k, 40 + sid, 1100.0).astype(np.float32)
        ids = torch.full((k,), sid, dtype=torch.int32, device="cuda")
        _check(sim, oracle_mod.Scene.from_workload(sc, bvh=False), ids, s, 50.0)


def test_nearest_zero_agents_and_far_outside(make_sim, oracle_mod, wl):
    """No agents is a no-op; agents far outside the scene's bounds still get
    the exact nearest point (the walk prunes nothing wrongly), or max_dist."""
    p = wl.params()
    sc = wl.room_scene()
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    from paper_2407_14783_b300.sim import to_soa
    out = sim.nearest_obstacle(torch.zeros((0,), dtype=torch.int32, device="cuda"),
                               to_soa(np.zeros((0, 17), np.float32)), 5.0)
    assert out[0].numel() == 0
    s = wl.spawn_states(sc, 6, 41, 1100.0).astype(np.float32)
    s[:, 0:3] += np.array([[40.0, 0, 0], [-35.0, 5, 0], [0, 60.0, 0], [0, 0, 25.0], [0, 0, -30.0], [70.0, 70.0, 70.0]],
                          np.float32)
    ids = torch.full((6,), sid, dtype=torch.int32, device="cuda")
    osc = oracle_mod.Scene.from_workload(sc, bvh=False)
    d = _check(sim, osc, ids, s, 500.0)
    assert d.min() > 10.0
    _check(sim, osc, ids, s, 20.0)
