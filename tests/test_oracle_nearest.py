"""Pins of the oracle's nearest-obstacle query (the distance module of Sec. III-B)."""
import numpy as np


def _scene(oracle_mod, v, f):
    f = np.asarray(f, np.int32)
    return oracle_mod.Scene(np.asarray(v, np.float32), f, np.zeros((f.shape[0], 3), np.uint8), bvh=False)


def test_triangle_regions(oracle_mod):
    """Face region: distance = height above the plane; vertex region: distance to
    the vertex; edge region: distance to the segment."""
    v = [[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.0, 2.0, 0.0]]
    sc = _scene(oracle_mod, v, [[0, 1, 2]])
    pts = np.array([[0.5, 0.5, 1.5],      # above the face
                    [-1.0, -2.0, 0.5],    # beyond vertex 0
                    [3.0, -0.5, 0.0],     # beyond vertex 1
                    [1.0, -1.0, 2.0],     # beyond edge 0-1
                    [2.0, 2.0, -1.0]])    # beyond edge 1-2
    d, q, t = sc.nearest(pts, 100.0)
    ref = [1.5, np.sqrt(1 + 4 + 0.25), np.sqrt(1 + 0.25), np.sqrt(1 + 4), np.sqrt(2 + 1)]
    assert np.allclose(d, ref, rtol=0, atol=1e-12)
    assert np.allclose(q[0], [0.5, 0.5, 0.0]) and np.allclose(q[1], v[0]) and np.allclose(q[2], v[1])
    assert np.allclose(q[3], [1.0, 0.0, 0.0]) and np.allclose(q[4], [1.0, 1.0, 0.0])
    assert np.all(t == 0)


def test_box_outside_closed_form(oracle_mod, wl):
    """Distance from an outside point to an axis-aligned box:
    sqrt(sum_j max(lo_j - p_j, 0, p_j - hi_j)^2)."""
    lo, hi = np.array([1.0, -2.0, 0.5]), np.array([3.0, 1.0, 2.5])
    v, f = wl.box_mesh(lo, hi)
    sc = _scene(oracle_mod, v, f)
    rng = np.random.default_rng(1)
    p = rng.uniform(-5, 7, (300, 3))
    outside = np.any((p < lo) | (p > hi), axis=1)
    p = p[outside]
    d, q, t = sc.nearest(p, 1e9)
    ref = np.sqrt(np.sum(np.maximum(np.maximum(lo - p, 0.0), p - hi) ** 2, axis=1))
    assert np.allclose(d, ref, rtol=0, atol=1e-9)
    assert np.allclose(np.linalg.norm(q - p, axis=1), d, atol=1e-9)


def test_room_inside_is_distance_to_nearest_wall(oracle_mod, wl):
    L = np.array([6.0, 5.0, 3.0])
    v, f = wl.box_mesh((0, 0, 0), L)
    sc = _scene(oracle_mod, v, f)
    p = np.random.default_rng(2).uniform(0.1, 1.0, (100, 3)) * L
    d, _, _ = sc.nearest(p, 1e9)
    assert np.allclose(d, np.minimum(p, L - p).min(axis=1), atol=1e-9)


def test_max_dist_and_sampling_bound(oracle_mod):
    """Beyond max_dist: id -1; the exact distance never exceeds the distance to any
    sampled point of the triangle and is within the sampling spacing of their minimum."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        tri = rng.normal(size=(3, 3))
        sc = _scene(oracle_mod, tri, [[0, 1, 2]])
        p = rng.normal(size=(1, 3)) * 2
        d, q, t = sc.nearest(p, 1e9)
        tri32 = tri.astype(np.float32).astype(np.float64)
        k = 200
        a, b = np.meshgrid(np.arange(k + 1) / k, np.arange(k + 1) / k)
        m = (a + b) <= 1
        pts = tri32[0] + a[m, None] * (tri32[1] - tri32[0]) + b[m, None] * (tri32[2] - tri32[0])
        samp = np.linalg.norm(pts - p[0], axis=1).min()
        assert d[0] <= samp + 1e-12
        edge = max(np.linalg.norm(tri32[i] - tri32[j]) for i in range(3) for j in range(3))
        assert samp - d[0] <= 2 * edge / k
        d2, q2, t2 = sc.nearest(p, d[0] * 0.5)
        assert t2[0] == -1 and d2[0] == d[0] * 0.5 and np.allclose(q2[0], p[0])
