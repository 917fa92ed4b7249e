"""Pins of the oracle's multi-agent (swarm) mode, Sec. III-B: the drones of a
scene see each other as boxes of the configured half extents about their body
origins, and collide as spheres.  Every expectation below comes from geometry
worked out by hand, not from the oracle's own slab formula."""
import math

import numpy as np
import pytest

HALF = (0.25, 0.18, 0.06)
DRONE_RGB = (250, 20, 30)


def _state(x, y, z, yaw=0.0):
    s = np.zeros(17)
    s[0:3] = (x, y, z)
    s[6] = math.cos(0.5 * yaw)
    s[9] = math.sin(0.5 * yaw)
    return s


def _empty_scene(oracle_mod):
    return oracle_mod.Scene(np.zeros((0, 3)), np.zeros((0, 3), np.int32), np.zeros((0, 3), np.uint8), bvh=False)


def _pixel_slopes(p):
    """Per column / row the lateral slopes u, v of the body-frame direction (1, -u, -v)."""
    th = math.tan(math.radians(p["fov_deg"]) / 2.0)
    W, H = p["width"], p["height"]
    u = (2.0 * np.arange(W) + 1.0 - W) / W * th
    v = (2.0 * np.arange(H) + 1.0 - H) / W * th
    return u, v


@pytest.mark.parametrize("yaw_b", [0.0, math.pi / 2, math.pi])
def test_drone_straight_ahead_closed_form(oracle_mod, wl, yaw_b):
    """Agent A at the origin looks along +x at drone B, D metres ahead.  Rays
    leave from a point on B's axis, so a ray enters B only through the face
    nearest A, at planar depth D - e_x, where (e_x, e_y) are B's half extents
    along world x and y (swapped by a 90-degree yaw).  A pixel is hit exactly
    when |u| (D - e_x) <= e_y and |v| (D - e_x) <= h_z."""
    p = wl.params()
    D = 1.2
    ex, ey = (HALF[1], HALF[0]) if abs(yaw_b - math.pi / 2) < 1e-9 else (HALF[0], HALF[1])
    st = np.stack([_state(0, 0, 1), _state(D, 0, 1, yaw_b)])
    r = _empty_scene(oracle_mod).render(p, st, use_bvh=False, swarm={"half": HALF, "rgb": DRONE_RGB})
    u, v = _pixel_slopes(p)
    near = D - ex
    inside = (np.abs(v)[:, None] * near <= HALF[2]) & (np.abs(u)[None, :] * near <= ey)
    # keep away from the silhouette, where the classification flags ties
    margin_u = np.abs(np.abs(u)[None, :] * near - ey)
    margin_v = np.abs(np.abs(v)[:, None] * near - HALF[2])
    clear = (margin_u > 1e-3) & (margin_v > 1e-3)
    a = 0
    assert inside.sum() > 20
    assert np.all(r["id"][a][inside & clear] == -2 - 1)
    assert np.allclose(r["depth"][a][inside & clear], near, rtol=0, atol=1e-12)
    assert np.all(r["rgb"][a][inside & clear] == np.array(DRONE_RGB, np.uint8))
    assert np.all(r["id"][a][~inside & clear] == -1)
    assert np.all(r["depth"][a][~inside & clear] == p["max_depth"])
    assert not r["tie"][a][clear].any()
    # B looks along +x (away from A) unless turned around, and never sees itself
    if yaw_b == 0.0:
        assert np.all(r["id"][1] == -1)


def test_mutual_view_at_equal_depth(oracle_mod, wl):
    """Two drones facing each other see one another at the same planar depth."""
    p = wl.params()
    D = 2.5
    st = np.stack([_state(0, 0, 1), _state(D, 0, 1, math.pi)])
    r = _empty_scene(oracle_mod).render(p, st, use_bvh=False, swarm={"half": HALF, "rgb": DRONE_RGB})
    c = p["width"] // 2
    for a, other in ((0, 1), (1, 0)):
        assert r["id"][a, c, c] == -2 - other
        assert abs(r["depth"][a, c, c] - (D - HALF[0])) < 1e-12


def test_single_agent_swarm_equals_plain_render(oracle_mod, wl):
    """A camera never sees its own drone: a one-agent swarm renders exactly
    like the parallel-agents mode."""
    p = wl.params()
    sc = wl.room_scene()
    st = wl.spawn_states(sc, 1, 12, 1100.0)
    o = oracle_mod.Scene.from_workload(sc)
    a = o.render(p, st)
    b = o.render(p, st, swarm={"half": HALF, "rgb": DRONE_RGB})
    for k in ("depth", "rgb", "id", "tie"):
        assert np.array_equal(a[k], b[k])


def test_drones_only_ever_occlude(oracle_mod, wl):
    """Adding drones can only bring hits closer: depth never grows, and every
    changed pixel shows a drone."""
    p = wl.params()
    sc = wl.room_scene()
    st = wl.spawn_states(sc, 12, 13, 1100.0)
    st[:, 0:3] = st[0, 0:3] + np.random.default_rng(3).uniform(-1.5, 1.5, (12, 3))   # a tight cluster
    st[:, 2] = np.clip(st[:, 2], 0.5, 3.5)
    o = oracle_mod.Scene.from_workload(sc)
    a = o.render(p, st)
    b = o.render(p, st, swarm={"half": HALF, "rgb": DRONE_RGB})
    assert np.all(b["depth"] <= a["depth"])
    changed = b["id"] != a["id"]
    assert changed.sum() > 100
    assert np.all(b["id"][changed & ~b["tie"]] <= -2)


def test_hit_point_lies_on_the_drone_surface_and_nothing_is_nearer(oracle_mod, wl):
    """For random poses: the reported point o + t d lies on drone j's box
    surface (max_k |p_k| / h_k = 1 in its body frame), and points of the ray
    before it lie outside every box."""
    p = wl.params(width=16, height=16)
    rng = np.random.default_rng(7)
    n = 6
    st = np.zeros((n, 17))
    st[:, 0:3] = rng.uniform(-1.0, 1.0, (n, 3))
    q = rng.normal(size=(n, 4))
    st[:, 6:10] = q / np.linalg.norm(q, axis=1, keepdims=True)
    r = _empty_scene(oracle_mod).render(p, st, use_bvh=False, swarm={"half": HALF, "rgb": DRONE_RGB})

    def rot(qq):
        w, x, y, z = qq
        return np.array([[w * w + x * x - y * y - z * z, 2 * (x * y - w * z), 2 * (x * z + w * y)],
                         [2 * (x * y + w * z), w * w - x * x + y * y - z * z, 2 * (y * z - w * x)],
                         [2 * (x * z - w * y), 2 * (y * z + w * x), w * w - x * x - y * y + z * z]])

    th = math.tan(math.radians(p["fov_deg"]) / 2.0)
    hits = 0
    for a in range(n):
        Ra = rot(st[a, 6:10])
        for row in range(16):
            for col in range(16):
                j = r["id"][a, row, col]
                if j >= -1 or r["tie"][a, row, col]:
                    continue
                j = -2 - j
                dB = np.array([1.0, -(2 * col + 1 - 16) / 16 * th, -(2 * row + 1 - 16) / 16 * th])
                d = Ra @ dB
                t = r["depth"][a, row, col]
                Rj = rot(st[j, 6:10])
                pt = Rj.T @ (st[a, 0:3] + t * d - st[j, 0:3])
                assert abs(np.max(np.abs(pt) / np.array(HALF)) - 1.0) < 1e-9
                for k in range(n):
                    if k == a:
                        continue
                    Rk = rot(st[k, 6:10])
                    if np.max(np.abs(Rk.T @ (st[a, 0:3] - st[k, 0:3])) / np.array(HALF)) <= 1.0:
                        continue          # camera inside box k: its hit is the exit, earlier points are inside
                    for s_ in np.linspace(1e-3, t * (1 - 1e-6), 40):
                        pk = Rk.T @ (st[a, 0:3] + s_ * d - st[k, 0:3])
                        assert np.max(np.abs(pk) / np.array(HALF)) > 1.0 - 1e-9
                hits += 1
    assert hits > 10


def test_proximity_on_a_line(oracle_mod):
    """Agents at x = 0, 1, 3: nearest distances 1, 1, 2; with radius 0.6 the
    first two collide (1 < 1.2), the third does not."""
    pos = np.array([[0, 0, 0], [1, 0, 0], [3, 0, 0]], float)
    dist, other, hits = oracle_mod.swarm_proximity(pos, 0.6)
    assert np.allclose(dist, [1, 1, 2]) and list(other) == [1, 0, 1] and list(hits) == [1, 1, 0]
    d1, o1, h1 = oracle_mod.swarm_proximity(pos[:1], 0.6)
    assert math.isinf(d1[0]) and o1[0] == -1 and h1[0] == 0


def test_proximity_equidistant_takes_lowest_index(oracle_mod):
    pos = np.array([[0, 0, 0], [0, 2, 0], [2, 0, 0], [0, 0, 2]], float)
    dist, other, hits = oracle_mod.swarm_proximity(pos, 2.0)
    assert dist[0] == 2.0 and other[0] == 1 and hits[0] == 3      # all three at 2 < 2 * 2.0
    dist, other, hits = oracle_mod.swarm_proximity(pos, 1.0)
    assert hits[0] == 0                                           # 2 < 2 * 1.0 is false


def test_swarm_views_equal_the_full_swarm_render(oracle_mod, wl):
    """Rendering chosen cameras of a swarm gives exactly those cameras' images
    of the full swarm render (the views form only selects cameras)."""
    p = wl.params(width=24, height=16)
    sc = wl.room_scene()
    osc = oracle_mod.Scene.from_workload(sc)
    rng = np.random.default_rng(3)
    st = wl.spawn_states(sc, 9, 12, 1100.0)
    st[:, 0:3] = st[0, 0:3] + rng.uniform(-1.0, 1.0, (9, 3))
    st[:, 2] = np.clip(st[:, 2], 0.6, 3.4)
    sw = {"half": (0.25, 0.18, 0.06), "rgb": (250, 20, 30)}
    full = osc.render(p, st, swarm=sw)
    pick = np.array([7, 2, 5])
    part = osc.render(p, st[pick], swarm={**sw, "states": st, "self": pick})
    for k in ("depth", "rgb", "id", "tie"):
        assert np.array_equal(part[k], full[k][pick]), k
    assert (part["id"] <= -2).any()
    # the oracle's own answers are admissible at its ambiguous pixels
    tie = np.flatnonzero(part["tie"].ravel())
    pix = tie if tie.size else np.arange(5)
    ok = osc.validate(p, st[pick], pix, part["id"].ravel()[pix], part["depth"].ravel()[pix].astype(np.float32),
                      swarm={**sw, "states": st, "self": pick})
    assert ok.all()
