"""Seeded synthetic inputs for the rollout-step hot path.

This module generates inputs only: quadrotor parameter values, triangle-mesh
scenes shaped like the paper's cluttered "stones in a garage" scene (Sec. IV-A,
0.15 obstacles per cubic metre), spawn states and command sequences.  It holds
none of the simulated method's arithmetic (no controller, dynamics, rotor model
or ray casting) and imports nothing from the CUDA path or from the oracle, so
both sides can consume the same inputs.

Randomness comes from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), evaluated counter-style with
numpy uint64 arithmetic so a stream is reproducible from (seed, draw index).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------
# Parameter values.  The paper names the model terms (Eq. 1-4) but prints none
# of the constants; these are the values this implementation adopts.  They are
# plain data: both the CUDA library and the oracle receive them as arguments.
# ----------------------------------------------------------------------------

DEFAULT_PARAMS: dict = {
    "mass": 1.0,                         # kg
    "J": (0.005, 0.005, 0.009),          # diagonal inertia, kg m^2
    "arm": 0.15,                         # rotor distance from the centre, m (X layout)
    "k": (0.0, 0.0, 2.0e-6),             # thrust polynomial k0, k1, k2 (Eq. 4)
    "c_lag": 1.0 / 0.03,                 # rotor time-decay constant c, 1/s (Eq. 4)
    "kappa": 0.016,                      # rotor drag torque / thrust ratio, m
    "rho": 1.225,                        # air density, kg/m^3 (Eq. 2)
    "Cd": (0.5, 0.5, 0.5),               # drag coefficients (Eq. 2)
    "area": (0.03, 0.03, 0.06),          # crossing areas, m^2 (Eq. 2)
    "omega_min": 0.0,                    # rotor speed limits, rad/s
    "omega_max": 2500.0,
    "a_max": 50.0,                       # mass-normalised thrust at u0 = +1, m/s^2
    "rate_max": (math.pi, math.pi, math.pi / 2.0),  # body-rate command scale, rad/s
    "K_rate": (20.0, 20.0, 10.0),        # body-rate loop gains, 1/s
    "g": 9.81,                           # gravity, m/s^2 (world z up)
    "dt": 0.02,                          # control step, s
    "n_sub": 1,                          # physics sub-steps per control step
    "integrator": 0,                     # 0 = RK4, 1 = explicit Euler
    "width": 64,                         # camera image size, pixels
    "height": 64,
    "fov_deg": 90.0,                     # horizontal and vertical field of view
    "max_depth": 10.0,                   # m; beyond this a ray is a miss
    "cam_off": (0.0, 0.0, 0.0),          # camera origin in the body frame, m
    "controller": 0,                     # 0 CTBR, 1 SRT, 2 LV (velocity + yaw), 3 PS (position + yaw)
    "K_pos": (4.0, 4.0, 6.0),            # LV / PS gains: position 1/s^2, velocity 1/s,
    "K_vel": (4.0, 4.0, 6.0),            # attitude 1/s^2, body rate 1/s
    "K_att": (150.0, 150.0, 40.0),
    "K_omega": (20.0, 20.0, 10.0),
}

# Rotor spin directions, rotor i at azimuth 45 + 90 i degrees.
ROTOR_SPIN = (1.0, -1.0, 1.0, -1.0)


def params(**overrides) -> dict:
    """Return a copy of DEFAULT_PARAMS with the given keys replaced."""
    p = dict(DEFAULT_PARAMS)
    for k, v in overrides.items():
        if k not in p:
            raise KeyError(f"unknown parameter {k!r}")
        p[k] = v
    return p


# ----------------------------------------------------------------------------
# SplitMix64
# ----------------------------------------------------------------------------

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """Output number ``index`` (0-based) of the SplitMix64 stream started at ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (np.asarray(index, dtype=np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Rng:
    """Sequential draws from one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.count = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.count, self.count + n, dtype=np.uint64)
        self.count += n
        return splitmix64(self.seed, idx)

    def uniform(self, lo=0.0, hi=1.0, size=1) -> np.ndarray:
        n = int(np.prod(size))
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return (lo + (hi - lo) * u).reshape(size)

    def log_uniform(self, lo, hi, size=1) -> np.ndarray:
        return np.exp(self.uniform(math.log(lo), math.log(hi), size))

    def integers(self, lo: int, hi: int, size=1) -> np.ndarray:
        """Uniform integers in [lo, hi)."""
        return (lo + np.floor(self.uniform(0.0, 1.0, size) * (hi - lo))).astype(np.int64)

    def bytes_u8(self, size) -> np.ndarray:
        n = int(np.prod(size))
        return (self.u64(n) >> np.uint64(56)).astype(np.uint8).reshape(size)


# ----------------------------------------------------------------------------
# Mesh primitives (indexed triangle lists, float64 vertices)
# ----------------------------------------------------------------------------

def box_mesh(lo, hi):
    """Axis-aligned box: 8 vertices, 12 triangles."""
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    v = np.array([[lo[0], lo[1], lo[2]], [hi[0], lo[1], lo[2]], [hi[0], hi[1], lo[2]], [lo[0], hi[1], lo[2]],
                  [lo[0], lo[1], hi[2]], [hi[0], lo[1], hi[2]], [hi[0], hi[1], hi[2]], [lo[0], hi[1], hi[2]]])
    f = np.array([[0, 2, 1], [0, 3, 2],      # z = lo
                  [4, 5, 6], [4, 6, 7],      # z = hi
                  [0, 1, 5], [0, 5, 4],      # y = lo
                  [3, 7, 6], [3, 6, 2],      # y = hi
                  [0, 4, 7], [0, 7, 3],      # x = lo
                  [1, 2, 6], [1, 6, 5]],     # x = hi
                 dtype=np.int64)
    return v, f


def cylinder_mesh(center, radius, height, segments=32):
    """Vertical cylinder: side quads split in two plus fan caps (4 * segments triangles)."""
    cx, cy, cz = center
    ang = 2.0 * np.pi * np.arange(segments) / segments
    ring = np.stack([cx + radius * np.cos(ang), cy + radius * np.sin(ang)], axis=1)
    z0, z1 = cz - 0.5 * height, cz + 0.5 * height
    bottom = np.column_stack([ring, np.full(segments, z0)])
    top = np.column_stack([ring, np.full(segments, z1)])
    v = np.vstack([bottom, top, [[cx, cy, z0], [cx, cy, z1]]])
    i = np.arange(segments)
    j = (i + 1) % segments
    cb, ct = 2 * segments, 2 * segments + 1
    side_a = np.stack([i, j, segments + j], axis=1)
    side_b = np.stack([i, segments + j, segments + i], axis=1)
    cap_b = np.stack([np.full(segments, cb), j, i], axis=1)
    cap_t = np.stack([np.full(segments, ct), segments + i, segments + j], axis=1)
    f = np.vstack([side_a, side_b, cap_b, cap_t]).astype(np.int64)
    return v, f


_ICO_CACHE: dict = {}


def _unit_icosphere(subdiv: int):
    if subdiv in _ICO_CACHE:
        return _ICO_CACHE[subdiv]
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
         [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
         [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]]
    f = [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
         [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
         [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]]
    verts = [np.array(p, float) / np.linalg.norm(p) for p in v]
    for _ in range(subdiv):
        mid = {}
        nf = []

        def midpoint(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                mid[key] = len(verts) - 1
            return mid[key]

        for a, b, c in f:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        f = nf
    out = (np.array(verts), np.array(f, dtype=np.int64))
    _ICO_CACHE[subdiv] = out
    return out


def icosphere_mesh(center, radius, subdiv=3):
    """Icosphere: 20 * 4**subdiv triangles with vertices on the sphere."""
    uv, f = _unit_icosphere(subdiv)
    return np.asarray(center, float) + radius * uv, f.copy()


def tessellated_plane(origin, axis_u, axis_v, nu, nv):
    """Rectangle origin + [0,1]axis_u + [0,1]axis_v split into nu*nv quads, 2 triangles each."""
    origin = np.asarray(origin, float)
    axis_u = np.asarray(axis_u, float)
    axis_v = np.asarray(axis_v, float)
    a = np.arange(nu + 1) / nu
    b = np.arange(nv + 1) / nv
    v = origin + a[:, None, None] * axis_u + b[None, :, None] * axis_v
    v = v.reshape(-1, 3)
    idx = lambda i, j: i * (nv + 1) + j
    f = []
    for i in range(nu):
        for j in range(nv):
            f.append([idx(i, j), idx(i + 1, j), idx(i + 1, j + 1)])
            f.append([idx(i, j), idx(i + 1, j + 1), idx(i, j + 1)])
    return v, np.array(f, dtype=np.int64)


# ----------------------------------------------------------------------------
# Scenes
# ----------------------------------------------------------------------------

@dataclass
class Scene:
    """An indexed triangle mesh with one uint8 RGB colour per triangle.

    ``verts`` float32 [V,3], ``tris`` int32 [T,3], ``rgb`` uint8 [T,3].
    ``room`` = (lo, hi) of the enclosing room; ``obstacles`` = object AABBs [K,2,3]
    (used by the spawn sampler for clearance).
    """
    verts: np.ndarray
    tris: np.ndarray
    rgb: np.ndarray
    room: tuple
    obstacles: np.ndarray
    seed: int = 0
    kinds: dict = field(default_factory=dict)

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


def _assemble(parts, rng: Rng, room, obstacles, seed, kinds) -> Scene:
    verts, tris = [], []
    off = 0
    for v, f in parts:
        verts.append(v)
        tris.append(f + off)
        off += v.shape[0]
    V = np.vstack(verts).astype(np.float32)
    T = np.vstack(tris).astype(np.int32)
    rgb = rng.bytes_u8((T.shape[0], 3))
    return Scene(V, T, rgb, room, np.asarray(obstacles, float).reshape(-1, 2, 3), seed, kinds)


def room_scene(size=(10.0, 10.0, 4.0), n_boxes=40, box_side=(0.2, 1.5), seed=1) -> Scene:
    """Closed room (12 triangles) with axis-aligned boxes of uniform side lengths."""
    rng = Rng(seed)
    L = np.asarray(size, float)
    parts = [box_mesh((0, 0, 0), L)]
    obstacles = []
    for _ in range(n_boxes):
        s = rng.uniform(box_side[0], box_side[1], 3)
        c = rng.uniform(0.0, 1.0, 3) * (L - s) + 0.5 * s
        lo, hi = c - 0.5 * s, c + 0.5 * s
        parts.append(box_mesh(lo, hi))
        obstacles.append([lo, hi])
    return _assemble(parts, rng, (np.zeros(3), L), obstacles, seed, {"box": n_boxes})


def cluttered_scene(n_objects=2000, size=(50.0, 50.0, 6.0), mix=(0.70, 0.25, 0.05),
                    obj_size=(0.1, 2.0), seed=2) -> Scene:
    """Procedural cluttered room: boxes, 32-segment cylinders and subdivision-3 icospheres.

    Counts of each kind are round(mix * n_objects) (boxes take the remainder);
    object sizes are log-uniform in ``obj_size``; centres are uniform with the
    object inside the room.
    """
    rng = Rng(seed)
    L = np.asarray(size, float)
    n_cyl = int(round(mix[1] * n_objects))
    n_sph = int(round(mix[2] * n_objects))
    n_box = n_objects - n_cyl - n_sph
    kinds_seq = [0] * n_box + [1] * n_cyl + [2] * n_sph
    parts = [box_mesh((0, 0, 0), L)]
    obstacles = []
    for kind in kinds_seq:
        if kind == 0:
            s = rng.log_uniform(obj_size[0], obj_size[1], 3)
            s = np.minimum(s, L)
            c = rng.uniform(0.0, 1.0, 3) * (L - s) + 0.5 * s
            lo, hi = c - 0.5 * s, c + 0.5 * s
            parts.append(box_mesh(lo, hi))
        elif kind == 1:
            d, h = rng.log_uniform(obj_size[0], obj_size[1], 2)
            r = 0.5 * d
            ext = np.array([d, d, h])
            c = rng.uniform(0.0, 1.0, 3) * (L - ext) + 0.5 * ext
            parts.append(cylinder_mesh(c, r, h))
            lo, hi = c - 0.5 * ext, c + 0.5 * ext
        else:
            d = float(rng.log_uniform(obj_size[0], obj_size[1], 1)[0])
            ext = np.full(3, d)
            c = rng.uniform(0.0, 1.0, 3) * (L - ext) + 0.5 * ext
            parts.append(icosphere_mesh(c, 0.5 * d))
            lo, hi = c - 0.5 * ext, c + 0.5 * ext
        obstacles.append([lo, hi])
    return _assemble(parts, rng, (np.zeros(3), L), obstacles, seed,
                     {"box": n_box, "cylinder": n_cyl, "sphere": n_sph})


def sized_scene(n_tris_target: int, seed: int, density=0.133, height=6.0) -> Scene:
    """Cluttered scene with about ``n_tris_target`` triangles at the given object density.

    Objects = (T - 12) / 104.4 (the mean triangles per object of the 70/25/5 mix);
    square room of side sqrt(objects / density / height).
    """
    n_obj = max(1, int(round((n_tris_target - 12) / 104.4)))
    side = math.sqrt(n_obj / density / height)
    return cluttered_scene(n_objects=n_obj, size=(side, side, height), seed=seed)


# ----------------------------------------------------------------------------
# Agents
# ----------------------------------------------------------------------------

STATE_DIM = 17   # x(3) v(3) q(4: w,x,y,z) Omega(3) omega_rotor(4)
CMD_DIM = 4      # normalised collective thrust, body-rate x, y, z


def _quat_from_euler(yaw, pitch, roll):
    cy, sy = np.cos(yaw / 2), np.sin(yaw / 2)
    cp, sp = np.cos(pitch / 2), np.sin(pitch / 2)
    cr, sr = np.cos(roll / 2), np.sin(roll / 2)
    w = cr * cp * cy + sr * sp * sy
    x = sr * cp * cy - cr * sp * sy
    y = cr * sp * cy + sr * cp * sy
    z = cr * cp * sy - sr * sp * cy
    return np.stack([w, x, y, z], axis=-1)


def spawn_states(scene: Scene, n: int, seed: int, omega0: float, clearance=0.3,
                 tilt=0.2, vel=0.5, rate=0.5) -> np.ndarray:
    """Agent states [n, 17] (float64) in the free space of ``scene``.

    Positions are uniform in the room, rejected when closer than ``clearance`` to a
    wall or to any obstacle AABB; yaw uniform, roll/pitch U(-tilt, tilt); linear
    and angular velocity U(-vel, vel) / U(-rate, rate); all four rotor speeds
    ``omega0``.
    """
    rng = Rng(seed)
    lo, hi = (np.asarray(a, float) for a in scene.room)
    obs = scene.obstacles
    out = np.zeros((n, STATE_DIM))
    got = 0
    tries = 0
    while got < n:
        tries += 1
        if tries > 1000:
            raise RuntimeError("spawn sampler could not find free space")
        m = max(64, 2 * (n - got))
        p = lo + clearance + rng.uniform(0.0, 1.0, (m, 3)) * (hi - lo - 2 * clearance)
        ok = np.ones(m, bool)
        if obs.shape[0]:
            for s in range(0, obs.shape[0], 512):
                o = obs[s:s + 512]
                inside = np.all((p[:, None, :] > o[None, :, 0, :] - clearance) &
                                (p[:, None, :] < o[None, :, 1, :] + clearance), axis=2)
                ok &= ~inside.any(axis=1)
        p = p[ok][: n - got]
        out[got:got + p.shape[0], 0:3] = p
        got += p.shape[0]
    yaw = rng.uniform(-math.pi, math.pi, n)
    pitch = rng.uniform(-tilt, tilt, n)
    roll = rng.uniform(-tilt, tilt, n)
    out[:, 6:10] = _quat_from_euler(yaw, pitch, roll)
    out[:, 3:6] = rng.uniform(-vel, vel, (n, 3))
    out[:, 10:13] = rng.uniform(-rate, rate, (n, 3))
    out[:, 13:17] = omega0
    return out


def uniform_commands(n_steps: int, n: int, seed: int) -> np.ndarray:
    """Commands [n_steps, n, 4] uniform in [-1, 1]."""
    return Rng(seed).uniform(-1.0, 1.0, (n_steps, n, CMD_DIM))


def hover_commands(n_steps: int, n: int, seed: int, u_thrust: float, thrust_jitter=0.1,
                   rate_range=1.0) -> np.ndarray:
    """Commands [n_steps, n, 4]: thrust u_thrust + U(-jitter, jitter), rates U(-r, r)."""
    rng = Rng(seed)
    u = np.empty((n_steps, n, CMD_DIM))
    u[..., 0] = u_thrust + rng.uniform(-thrust_jitter, thrust_jitter, (n_steps, n))
    u[..., 1:] = rng.uniform(-rate_range, rate_range, (n_steps, n, 3))
    return u


def zipf_partition(n_agents: int, n_scenes: int, alpha: float, seed: int) -> np.ndarray:
    """Agents per scene: Zipf(alpha) weights over a seeded random ranking of scenes,
    at least one agent per scene, largest-remainder rounding.  Returns int64 [n_scenes]."""
    rng = Rng(seed)
    rank_of = np.argsort(rng.uniform(0.0, 1.0, n_scenes))
    w = 1.0 / np.power(np.arange(1, n_scenes + 1, dtype=float), alpha)
    w = w[np.argsort(rank_of)]
    w /= w.sum()
    base = np.ones(n_scenes, dtype=np.int64)
    rest = n_agents - n_scenes
    if rest < 0:
        raise ValueError("need at least one agent per scene")
    share = w * rest
    cnt = np.floor(share).astype(np.int64)
    left = rest - int(cnt.sum())
    order = np.argsort(-(share - cnt), kind="stable")
    cnt[order[:left]] += 1
    return base + cnt


def goal_points(scene: Scene, n: int, seed: int, clearance=0.3) -> np.ndarray:
    """Goal positions [n, 3] in free space (same sampler as the spawn positions)."""
    return spawn_states(scene, n, seed, 0.0, clearance)[:, 0:3].copy()


def poisson_requests(rate_hz: float, duration_s: float, n_scenes: int, seed: int,
                     agents=(1, 1024), steps=(1, 16)):
    """Poisson arrival times with per-request (scene, agents, steps).

    Returns a list of dicts sorted by arrival time: scene U{0..n_scenes-1},
    agents round(log-uniform[agents]), steps U{steps[0]..steps[1]}.
    """
    rng = Rng(seed)
    out = []
    t = 0.0
    while True:
        t += -math.log(1.0 - float(rng.uniform(0.0, 1.0, 1)[0])) / rate_hz
        if t >= duration_s:
            break
        sc = int(rng.integers(0, n_scenes, 1)[0])
        na = int(round(float(rng.log_uniform(agents[0], agents[1], 1)[0])))
        ns = int(rng.integers(steps[0], steps[1] + 1, 1)[0])
        out.append({"t": t, "scene": sc, "agents": na, "steps": ns})
    return out
