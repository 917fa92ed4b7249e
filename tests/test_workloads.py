"""Checks of the seeded input generators (no method arithmetic lives there)."""
import numpy as np


def test_splitmix64_reference_outputs(wl):
    """First two outputs of SplitMix64 started from state 0, as produced by the
    published reference generator (Steele, Lea, Flood 2014; Vigna's splitmix64.c)."""
    out = wl.splitmix64(0, np.array([0, 1]))
    assert int(out[0]) == 0xE220A8397B1DCDAF
    assert int(out[1]) == 0x6E789E6AA1B965F4


def test_scene_sizes(wl):
    """Config sizes: tiny room 12 + 40 * 12 = 492 triangles; the large cluttered
    room 12 + 1400 * 12 + 500 * 128 + 100 * 1280 = 208,812 triangles."""
    a = wl.room_scene()
    assert a.n_tris == 492 and a.rgb.shape == (492, 3) and a.verts.dtype == np.float32
    b = wl.cluttered_scene()
    assert b.n_tris == 208812
    assert b.kinds == {"box": 1400, "cylinder": 500, "sphere": 100}
    assert np.all(b.tris >= 0) and np.all(b.tris < b.verts.shape[0])
    lo, hi = b.room
    assert np.all(b.verts >= lo - 1e-4) and np.all(b.verts <= hi + 1e-4)


def test_determinism(wl):
    a1, a2 = wl.cluttered_scene(n_objects=50, seed=9), wl.cluttered_scene(n_objects=50, seed=9)
    assert np.array_equal(a1.verts, a2.verts) and np.array_equal(a1.rgb, a2.rgb)
    s1 = wl.spawn_states(a1, 10, 4, 1000.0)
    s2 = wl.spawn_states(a2, 10, 4, 1000.0)
    assert np.array_equal(s1, s2)


def test_spawn_clearance(wl):
    sc = wl.cluttered_scene(n_objects=300, size=(20.0, 20.0, 6.0), seed=3)
    s = wl.spawn_states(sc, 200, 5, 1000.0)
    p = s[:, 0:3]
    lo, hi = sc.room
    assert np.all(p > lo + 0.3) and np.all(p < hi - 0.3)
    o = sc.obstacles
    inside = np.all((p[:, None, :] > o[None, :, 0, :] - 0.3) & (p[:, None, :] < o[None, :, 1, :] + 0.3), axis=2)
    assert not inside.any()
    assert np.allclose(np.linalg.norm(s[:, 6:10], axis=1), 1.0)


def test_zipf_partition(wl):
    c = wl.zipf_partition(4096, 64, 1.1, 7)
    assert c.sum() == 4096 and c.min() >= 1 and c.shape == (64,)
    assert c.max() > 10 * np.median(c)


def test_poisson_requests(wl):
    r = wl.poisson_requests(2000.0, 0.5, 32, 5)
    assert 800 < len(r) < 1200
    assert all(1 <= q["agents"] <= 1024 and 1 <= q["steps"] <= 16 for q in r)
    ts = [q["t"] for q in r]
    assert ts == sorted(ts)
