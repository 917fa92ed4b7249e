"""Pins of the FP64 oracle's renderer (Sec. III-B: depth and colour sensors)
against analytic geometry and brute force.

The camera reading under test: camera at the body origin looking along body
+x, image right = body -y, image down = body -z, pixel centres at +0.5, 90
degree field of view, depth = distance along the optical axis.
"""
import math

import numpy as np
import pytest


def _state(pos, q=(1.0, 0.0, 0.0, 0.0)):
    s = np.zeros((1, 17))
    s[0, 0:3] = pos
    s[0, 6:10] = np.asarray(q, float) / np.linalg.norm(q)
    return s


def _quat_axis_angle(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    return np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * axis])


def _rotmat(q):
    """Rotation matrix of a unit quaternion via the axis-angle (Rodrigues) form."""
    q = np.asarray(q, float) / np.linalg.norm(q)
    ang = 2.0 * math.atan2(np.linalg.norm(q[1:]), q[0])
    if ang == 0.0:
        return np.eye(3)
    k = q[1:] / np.linalg.norm(q[1:])
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def _pixel_dirs_world(q, W=64, H=64, fov=90.0):
    """World ray directions [H, W, 3] built from the pinhole model by hand."""
    f = 1.0 / math.tan(math.radians(fov) / 2)       # focal length in half-widths
    cols = (np.arange(W) + 0.5) / W * 2 - 1         # -1 .. 1 left to right
    rows = (np.arange(H) + 0.5) / H * 2 - 1         # -1 .. 1 top to bottom
    d = np.zeros((H, W, 3))
    d[..., 0] = 1.0
    d[..., 1] = -cols[None, :] / f
    d[..., 2] = -rows[:, None] / f
    return d @ _rotmat(q).T


def _scene(oracle_mod, verts, tris, rgb=None, bvh=True):
    tris = np.asarray(tris, np.int32)
    if rgb is None:
        rgb = (np.arange(tris.shape[0] * 3) % 251).astype(np.uint8).reshape(-1, 3)
    return oracle_mod.Scene(np.asarray(verts, np.float32), tris, rgb, bvh)


def test_frontal_plane_constant_depth(oracle_mod, wl):
    """A tessellated plane x = d in front of a level camera: planar depth is d at
    every pixel, and the triangle hit is the one of the tessellation cell that
    contains the analytic hit point."""
    d = 4.0
    nu = nv = 8
    v, f = wl.tessellated_plane((d, -20.0, -20.0), (0, 40.0, 0), (0, 0, 40.0), nu, nv)
    sc = _scene(oracle_mod, v, f)
    p = wl.params()
    out = sc.render(p, _state((0, 0, 0)))
    assert np.abs(out["depth"] - d).max() < 1e-12
    dirs = _pixel_dirs_world((1, 0, 0, 0))
    hit = d * dirs[..., 1:] / dirs[..., 0:1]         # (y, z) of the hit point
    a = (hit[..., 0] + 20.0) / 40.0 * nu
    b = (hit[..., 1] + 20.0) / 40.0 * nv
    i, j = np.floor(a).astype(int), np.floor(b).astype(int)
    fa, fb = a - i, b - j
    upper = fb > fa                                   # above the cell diagonal
    expect = 2 * (i * nv + j) + upper.astype(int)
    clear = (np.abs(fa - fb) > 1e-6) & (fa > 1e-6) & (fb > 1e-6)
    assert np.array_equal(out["id"][0][clear], expect[clear])
    assert not out["tie"][0][clear].any()


def test_tilted_plane_depth_formula(oracle_mod, wl):
    """Rotated camera, tilted plane x + 2y - z = 6 tessellated on integer vertices
    (exact in float32): t = (6 - n.o) / (n.d_world) for every ray that meets the
    patch within range; rays that do not are misses."""
    n = np.array([1.0, 2.0, -1.0])
    U = np.array([16.0, -8.0, 0.0])
    V = np.array([8.0, 0.0, 8.0])
    origin = np.array([-6.0, 4.0, -4.0])
    assert n @ U == 0 and n @ V == 0 and n @ origin == 6.0
    v, f = wl.tessellated_plane(origin, U, V, 8, 8)
    sc = _scene(oracle_mod, v, f)
    p = wl.params()
    q = _quat_axis_angle((0.2, -0.4, 1.0), 0.5)
    o = np.array([0.5, -0.2, 1.0])
    out = sc.render(p, _state(o, q))
    dirs = _pixel_dirs_world(q)
    t = (6.0 - n @ o) / (dirs @ n)
    X = o + t[..., None] * dirs - origin
    G = np.array([[U @ U, U @ V], [U @ V, V @ V]])
    ab = np.linalg.solve(G, np.stack([X @ U, X @ V], axis=-1)[..., None])[..., 0]
    inside = np.all((ab > 1e-6) & (ab < 1 - 1e-6), axis=-1)
    outside = np.any((ab < -1e-6) | (ab > 1 + 1e-6), axis=-1)
    ok = inside & (t > 0) & (t <= p["max_depth"] * (1 - 1e-9))
    miss = outside | (t <= 0) | (t > p["max_depth"] * (1 + 1e-9))
    assert ok.mean() > 0.2 and miss.mean() > 0.05
    assert np.abs(out["depth"][0][ok] - t[ok]).max() < 1e-12 * p["max_depth"]
    assert np.all(out["depth"][0][miss] == p["max_depth"])
    assert np.all(out["id"][0][miss] == -1)


def test_box_room_from_inside(oracle_mod, wl):
    """Inside a closed axis-aligned room every pixel sees the nearest of the six
    wall planes along its ray; each face's two triangles share a colour, so the
    colour image is exact too."""
    L = np.array([6.0, 5.0, 3.0])
    v, f = wl.box_mesh((0, 0, 0), L)
    face_rgb = np.array([[10, 0, 0], [20, 0, 0], [0, 30, 0], [0, 40, 0], [0, 0, 50], [0, 0, 60]], np.uint8)
    rgb = np.repeat(face_rgb, 2, axis=0)
    sc = _scene(oracle_mod, v, f, rgb)
    p = wl.params()
    rng = np.random.default_rng(3)
    for trial in range(6):
        o = rng.uniform(0.5, 1.0, 3) * L * rng.uniform(0.3, 0.9)
        q = _quat_axis_angle(rng.normal(size=3), rng.uniform(0, math.pi))
        out = sc.render(p, _state(o, q))
        dirs = _pixel_dirs_world(q)
        ts = np.full(dirs.shape[:2] + (6,), np.inf)
        for ax in range(3):
            dd = dirs[..., ax]
            with np.errstate(divide="ignore"):
                t_lo = (0.0 - o[ax]) / dd
                t_hi = (L[ax] - o[ax]) / dd
            ts[..., 2 * ax] = np.where(t_lo > 0, t_lo, np.inf)
            ts[..., 2 * ax + 1] = np.where(t_hi > 0, t_hi, np.inf)
        tmin = ts.min(axis=2)
        which = ts.argmin(axis=2)   # 0:x=0 1:x=L 2:y=0 3:y=L 4:z=0 5:z=L
        # mesh face order: z=lo, z=hi, y=lo, y=hi, x=lo, x=hi
        face_of = np.array([4, 5, 2, 3, 0, 1])[which]
        expect_depth = np.where(tmin <= p["max_depth"], tmin, p["max_depth"])
        assert np.abs(out["depth"][0] - expect_depth).max() < 1e-9
        clear = ~out["tie"][0]
        assert clear.mean() > 0.95
        hit = tmin <= p["max_depth"]
        assert np.array_equal(out["id"][0][clear & hit] // 2, face_of[clear & hit])
        assert np.array_equal(out["rgb"][0][clear & hit], face_rgb[face_of[clear & hit]])


def test_icosphere_between_inner_and_outer_sphere(oracle_mod, wl):
    """An icosphere has vertices on the sphere of radius r and faces no closer than
    r_in to its centre: rays that miss the outer sphere miss the mesh, rays that
    hit the inner sphere hit the mesh, and every hit depth lies between the
    first crossings of the two spheres."""
    c = np.array([5.0, 0.3, -0.2])
    r = 1.5
    v, f = wl.icosphere_mesh(c, r, 3)
    v32 = v.astype(np.float32).astype(np.float64)
    n = np.cross(v32[f[:, 1]] - v32[f[:, 0]], v32[f[:, 2]] - v32[f[:, 0]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    r_in = np.min(np.abs(np.einsum("ij,ij->i", n, v32[f[:, 0]] - c)))
    r_out = np.max(np.linalg.norm(v32 - c, axis=1))
    sc = _scene(oracle_mod, v, f)
    p = wl.params()
    q = _quat_axis_angle((0, 0, 1), 0.05)
    o = np.zeros(3)
    out = sc.render(p, _state(o, q))
    d = _pixel_dirs_world(q)

    def first_cross(rad):
        a = np.sum(d * d, axis=2)
        b = 2 * np.sum(d * (o - c), axis=2)
        cc = np.sum((o - c) ** 2) - rad * rad
        disc = b * b - 4 * a * cc
        t = np.where(disc >= 0, (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a), np.inf)
        return t, disc

    t_out, disc_out = first_cross(r_out)
    t_in, disc_in = first_cross(r_in)
    hit = out["id"][0] >= 0
    margin = 1e-9
    assert not np.any(hit & (disc_out < -margin))
    assert np.all(hit[disc_in > margin])
    dep = out["depth"][0]
    assert np.all(dep[hit] >= t_out[hit] - 1e-9)
    inner = hit & (disc_in > 0)
    assert np.all(dep[inner] <= t_in[inner] + 1e-9)
    assert hit.mean() > 0.05


@pytest.mark.parametrize("seed", range(8))
def test_bvh_equals_brute_force_small_random_meshes(oracle_mod, wl, seed):
    """The oracle's median-split BVH returns exactly the brute-force answer
    (depth, id, colour and ambiguity flag) on random 1-64-triangle meshes."""
    rng = np.random.default_rng(100 + seed)
    nt = int(rng.integers(1, 65))
    v = rng.uniform(-3, 3, (3 * nt, 3)) + np.array([4.0, 0, 0])
    f = np.arange(3 * nt).reshape(nt, 3)
    rgb = rng.integers(0, 256, (nt, 3)).astype(np.uint8)
    a = _scene(oracle_mod, v, f, rgb, bvh=True)
    p = wl.params(width=32, height=24)
    st = np.zeros((3, 17))
    st[:, 0:3] = rng.uniform(-1, 1, (3, 3))
    for k in range(3):
        st[k, 6:10] = _quat_axis_angle(rng.normal(size=3), rng.uniform(0, 0.6))
    r1 = a.render(p, st, use_bvh=True)
    r2 = a.render(p, st, use_bvh=False)
    for key in r1:
        assert np.array_equal(r1[key], r2[key]), key


def test_bvh_equals_brute_force_room_scene(oracle_mod, wl):
    """Same on the 492-triangle room scene with 4 spawned agents."""
    scn = wl.room_scene()
    sc = oracle_mod.Scene.from_workload(scn)
    p = wl.params()
    st = wl.spawn_states(scn, 4, 11, 1100.0)
    r1 = sc.render(p, st, use_bvh=True)
    r2 = sc.render(p, st, use_bvh=False)
    for key in r1:
        assert np.array_equal(r1[key], r2[key]), key
    assert r1["tie"].mean() < 0.01


def test_ambiguity_and_validator(oracle_mod, wl):
    """The validator accepts the oracle's own answers, rejects another triangle,
    a miss where a definite hit exists, and a depth off by 1e-3 relative."""
    scn = wl.room_scene()
    sc = oracle_mod.Scene.from_workload(scn)
    p = wl.params()
    st = wl.spawn_states(scn, 2, 12, 1100.0)
    r = sc.render(p, st)
    ids = r["id"].reshape(-1)
    dep = r["depth"].reshape(-1).astype(np.float32)
    pix = np.arange(ids.size)
    clear = ~r["tie"].reshape(-1)
    assert sc.validate(p, st, pix[clear], ids[clear], dep[clear]).all()
    hit = clear & (ids >= 0)
    sel = pix[hit][:200]
    wrong = (ids[sel] + 1) % scn.n_tris
    assert not sc.validate(p, st, sel, wrong, dep[sel]).any()
    assert not sc.validate(p, st, sel, np.full(sel.size, -1), np.full(sel.size, p["max_depth"], np.float32)).any()
    assert not sc.validate(p, st, sel, ids[sel], dep[sel] * np.float32(1.001)).any()


def test_shared_edge_is_ambiguous(oracle_mod, wl):
    """A ray through the diagonal shared by two triangles of one quad hits both at
    the same depth: the pixel is flagged ambiguous and either id validates."""
    v = np.array([[3.0, -2, -2], [3.0, 2, -2], [3.0, 2, 2], [3.0, -2, 2]])
    # the diagonal y = z of the quad contains the hit points of pixels (0,0) and (1,1)
    f = np.array([[0, 1, 2], [0, 2, 3]])
    sc = _scene(oracle_mod, v, f)
    p = wl.params(width=2, height=2)
    st = _state((0, 0, 0))
    r = sc.render(p, st)
    d = _pixel_dirs_world((1, 0, 0, 0), 2, 2)
    on_diag = np.isclose(d[..., 1], d[..., 2])
    assert on_diag.sum() == 2 and np.all(r["tie"][0][on_diag])
    assert not np.any(r["tie"][0][~on_diag])
    for k in np.flatnonzero(on_diag.reshape(-1)):
        for tid in (0, 1):
            ok = sc.validate(p, st, np.array([k]), np.array([tid]), np.array([3.0], np.float32))
            assert ok.all()


def test_ambiguous_fraction_large_scene(oracle_mod, wl):
    """On the 208,812-triangle cluttered room the ambiguous pixels stay below 1%."""
    scn = wl.cluttered_scene()
    sc = oracle_mod.Scene.from_workload(scn)
    p = wl.params()
    st = wl.spawn_states(scn, 16, 3, 1100.0)
    r = sc.render(p, st)
    assert r["tie"].mean() < 0.01
    assert 0.01 < (r["id"] < 0).mean() < 0.5


def test_traversal_counts_of_a_single_leaf_and_a_split(oracle_mod, wl):
    """The oracle's walk statistic: a mesh of at most 4 triangles is one leaf, so
    every ray visits no internal node and tests exactly those triangles; a scene
    behind the camera (all rays miss) visits only the root of its tree."""
    p = wl.params(width=8, height=6)
    s = np.zeros((2, 17))
    s[:, 6] = 1.0
    s[1, 0:3] = (0.3, -0.2, 0.1)
    v = np.array([[3.0, -1.0, -1.0], [3.0, 1.5, -1.0], [3.0, 0.0, 2.0], [4.0, 0.0, 0.0], [4.0, 1.0, 0.0]])
    one = oracle_mod.Scene(v, [[0, 1, 2], [1, 3, 4], [0, 3, 4]], [[1, 2, 3]] * 3)
    c = one.traversal_counts(p, s)
    assert c == {"nodes": 0.0, "tris": 3.0}
    bv, bf = wl.box_mesh((-8.0, -1.0, -1.0), (-6.0, 1.0, 1.0))     # 12 triangles behind the camera
    behind = oracle_mod.Scene(bv, bf, np.zeros((12, 3), np.uint8))
    c = behind.traversal_counts(p, s)
    assert c == {"nodes": 1.0, "tris": 0.0}
