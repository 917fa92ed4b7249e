"""FP64 CPU oracle for the VisFly rollout-step hot path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the package smoke
check and by the benchmark's CPU-baseline leg, never by the product library.
The C++ source (``oracle.cpp``) shares no code, header or constant with the
CUDA path; every parameter value arrives as an argument.

Arrays cross this wrapper in the oracle's own layout: agent-major
``[n, 17]`` states, ``[n, 4]`` commands, ``[T, n, 4]`` command sequences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (g++ -O2 -fopenmp)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double), ("J", ctypes.c_double * 3), ("arm", ctypes.c_double),
        ("k", ctypes.c_double * 3), ("c_lag", ctypes.c_double), ("kappa", ctypes.c_double),
        ("rho", ctypes.c_double), ("Cd", ctypes.c_double * 3), ("area", ctypes.c_double * 3),
        ("omega_min", ctypes.c_double), ("omega_max", ctypes.c_double), ("a_max", ctypes.c_double),
        ("rate_max", ctypes.c_double * 3), ("K_rate", ctypes.c_double * 3), ("g", ctypes.c_double),
        ("dt", ctypes.c_double), ("n_sub", ctypes.c_int32), ("integrator", ctypes.c_int32),
        ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fov_deg", ctypes.c_double),
        ("max_depth", ctypes.c_double), ("cam_off", ctypes.c_double * 3), ("controller", ctypes.c_int32),
        ("K_pos", ctypes.c_double * 3), ("K_vel", ctypes.c_double * 3), ("K_att", ctypes.c_double * 3),
        ("K_omega", ctypes.c_double * 3),
    ]


def make_params(p: dict) -> OracleParams:
    o = OracleParams()
    for name, ctype in OracleParams._fields_:
        v = p[name]
        if hasattr(ctype, "_length_"):
            setattr(o, name, ctype(*[float(x) for x in v]))
        elif ctype is ctypes.c_int32:
            setattr(o, name, int(v))
        else:
            setattr(o, name, float(v))
    return o


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER
            dp, i64, vp = P(ctypes.c_double), ctypes.c_int64, ctypes.c_void_p
            L.oracle_step.argtypes = [P(OracleParams), i64, dp, dp, dp]
            L.oracle_rollout.argtypes = [P(OracleParams), i64, i64, dp, dp, dp]
            L.oracle_step_vjp.argtypes = [P(OracleParams), i64, dp, dp, dp, dp, dp]
            L.oracle_rollout_loss_grad.argtypes = [P(OracleParams), i64, i64, dp, dp, dp, ctypes.c_double,
                                                   dp, dp, dp]
            L.oracle_scene_create.restype = vp
            L.oracle_scene_create.argtypes = [dp, i64, P(ctypes.c_int32), i64, P(ctypes.c_uint8), ctypes.c_int]
            L.oracle_scene_destroy.argtypes = [vp]
            L.oracle_scene_bvh_nodes.restype = i64
            L.oracle_scene_bvh_nodes.argtypes = [vp]
            L.oracle_traversal_counts.argtypes = [vp, P(OracleParams), i64, dp, dp]
            L.oracle_render.argtypes = [vp, P(OracleParams), i64, dp, ctypes.c_int, dp, P(ctypes.c_uint8),
                                        P(ctypes.c_int32), P(ctypes.c_uint8)]
            L.oracle_validate.argtypes = [vp, P(OracleParams), i64, dp, i64, P(ctypes.c_int64),
                                          P(ctypes.c_int32), P(ctypes.c_float), P(ctypes.c_uint8)]
            L.oracle_render_swarm.argtypes = [vp, P(OracleParams), i64, dp, ctypes.c_int, dp, P(ctypes.c_uint8), dp,
                                              P(ctypes.c_uint8), P(ctypes.c_int32), P(ctypes.c_uint8)]
            L.oracle_validate_swarm.argtypes = [vp, P(OracleParams), i64, dp, dp, i64, P(ctypes.c_int64),
                                                P(ctypes.c_int32), P(ctypes.c_float), P(ctypes.c_uint8)]
            L.oracle_render_swarm_views.argtypes = [vp, P(OracleParams), i64, dp, P(ctypes.c_int64), i64, dp,
                                                    ctypes.c_int, dp, P(ctypes.c_uint8), dp, P(ctypes.c_uint8),
                                                    P(ctypes.c_int32), P(ctypes.c_uint8)]
            L.oracle_validate_swarm_views.argtypes = [vp, P(OracleParams), i64, dp, P(ctypes.c_int64), i64, dp, dp,
                                                      i64, P(ctypes.c_int64), P(ctypes.c_int32), P(ctypes.c_float),
                                                      P(ctypes.c_uint8)]
            L.oracle_swarm_proximity.argtypes = [i64, dp, ctypes.c_double, dp, P(ctypes.c_int32), P(ctypes.c_int32)]
            L.oracle_num_threads.restype = ctypes.c_int
            L.oracle_nearest.argtypes = [vp, i64, dp, ctypes.c_double, dp, dp, P(ctypes.c_int32)]
            L.oracle_point_triangle.argtypes = [vp, i64, dp, P(ctypes.c_int32), dp]
            _lib = L
        return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def step(p: dict, state: np.ndarray, cmd: np.ndarray) -> np.ndarray:
    """One control step: state [n,17], cmd [n,4] -> new state [n,17]."""
    state, cmd = _f64(state), _f64(cmd)
    n = state.shape[0]
    out = np.empty_like(state)
    rc = lib().oracle_step(ctypes.byref(make_params(p)), n, _ptr(state, ctypes.c_double),
                           _ptr(cmd, ctypes.c_double), _ptr(out, ctypes.c_double))
    if rc:
        raise ValueError(f"oracle_step failed ({rc})")
    return out


def rollout(p: dict, state0: np.ndarray, cmds: np.ndarray) -> np.ndarray:
    """T steps: state0 [n,17], cmds [T,n,4] -> states [T+1,n,17]."""
    state0, cmds = _f64(state0), _f64(cmds)
    T, n = cmds.shape[0], state0.shape[0]
    out = np.empty((T + 1, n, 17))
    rc = lib().oracle_rollout(ctypes.byref(make_params(p)), n, T, _ptr(state0, ctypes.c_double),
                              _ptr(cmds, ctypes.c_double), _ptr(out, ctypes.c_double))
    if rc:
        raise ValueError(f"oracle_rollout failed ({rc})")
    return out


def step_vjp(p: dict, state: np.ndarray, cmd: np.ndarray, g_out: np.ndarray):
    """Vector-Jacobian product of one step: returns (g_state [n,17], g_cmd [n,4])."""
    state, cmd, g_out = _f64(state), _f64(cmd), _f64(g_out)
    n = state.shape[0]
    gs = np.empty((n, 17))
    gc = np.empty((n, 4))
    rc = lib().oracle_step_vjp(ctypes.byref(make_params(p)), n, _ptr(state, ctypes.c_double),
                               _ptr(cmd, ctypes.c_double), _ptr(g_out, ctypes.c_double),
                               _ptr(gs, ctypes.c_double), _ptr(gc, ctypes.c_double))
    if rc:
        raise ValueError(f"oracle_step_vjp failed ({rc})")
    return gs, gc


def rollout_loss_grad(p: dict, state0, cmds, goals, lam: float):
    """Loss per agent and its gradient w.r.t. state0 [n,17] and cmds [T,n,4]."""
    state0, cmds, goals = _f64(state0), _f64(cmds), _f64(goals)
    T, n = cmds.shape[0], state0.shape[0]
    loss = np.empty(n)
    gs = np.empty((n, 17))
    gc = np.empty((T, n, 4))
    rc = lib().oracle_rollout_loss_grad(ctypes.byref(make_params(p)), n, T, _ptr(state0, ctypes.c_double),
                                        _ptr(cmds, ctypes.c_double), _ptr(goals, ctypes.c_double), float(lam),
                                        _ptr(loss, ctypes.c_double), _ptr(gs, ctypes.c_double),
                                        _ptr(gc, ctypes.c_double))
    if rc:
        raise ValueError(f"oracle_rollout_loss_grad failed ({rc})")
    return loss, gs, gc


def rollout_loss(states: np.ndarray, cmds: np.ndarray, goals: np.ndarray, lam: float) -> np.ndarray:
    """Loss per agent from a trajectory states [T+1,n,17] (the formula of oracle_rollout_loss_grad)."""
    T = cmds.shape[0]
    e = states[1:, :, 0:3] - goals[None]
    return (e * e).sum(axis=(0, 2)) / T + lam * (cmds * cmds).sum(axis=(0, 2)) / T


class Scene:
    """Oracle-side copy of a mesh, optionally with its own median-split BVH."""

    def __init__(self, verts, tris, rgb, bvh: bool = True):
        v = _f64(np.asarray(verts, dtype=np.float32))  # the float32 values both sides see
        t = np.ascontiguousarray(np.asarray(tris, dtype=np.int32))
        c = np.ascontiguousarray(np.asarray(rgb, dtype=np.uint8))
        self._keep = (v, t, c)
        self.n_tris = t.shape[0]
        self.handle = lib().oracle_scene_create(_ptr(v, ctypes.c_double), v.shape[0], _ptr(t, ctypes.c_int32),
                                                t.shape[0], _ptr(c, ctypes.c_uint8), 1 if bvh else 0)
        if not self.handle:
            raise ValueError("oracle_scene_create failed")
        self.bvh = bvh

    @classmethod
    def from_workload(cls, scene, bvh: bool = True):
        return cls(scene.verts, scene.tris, scene.rgb, bvh)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            lib().oracle_scene_destroy(h)
            self.handle = None

    def render(self, p: dict, states: np.ndarray, use_bvh: bool | None = None, swarm: dict | None = None):
        """Returns dict depth [n,H,W] f64, rgb [n,H,W,3] u8, id [n,H,W] i32, tie [n,H,W] bool.

        swarm = {"half": (hx, hy, hz), "rgb": (r, g, b)} renders the n agents as
        one swarm: each sees the other drones (id -2 - j for drone j).  With
        swarm["states"] ([m, 17], the whole swarm) and swarm["self"] ([n], the
        swarm index of each rendered agent) only the n given cameras are
        rendered, each seeing every other drone of the swarm."""
        states = _f64(states)
        n = states.shape[0]
        H, W = int(p["height"]), int(p["width"])
        depth = np.empty((n, H, W))
        rgb = np.empty((n, H, W, 3), np.uint8)
        hid = np.empty((n, H, W), np.int32)
        tie = np.empty((n, H, W), np.uint8)
        ub = self.bvh if use_bvh is None else use_bvh
        if swarm is None:
            rc = lib().oracle_render(self.handle, ctypes.byref(make_params(p)), n, _ptr(states, ctypes.c_double),
                                     1 if ub else 0, _ptr(depth, ctypes.c_double), _ptr(rgb, ctypes.c_uint8),
                                     _ptr(hid, ctypes.c_int32), _ptr(tie, ctypes.c_uint8))
        elif "states" in swarm:
            half = np.ascontiguousarray(swarm["half"], dtype=np.float64)
            col = np.ascontiguousarray(swarm.get("rgb", (0, 0, 0)), dtype=np.uint8)
            allst = _f64(swarm["states"])
            me = np.ascontiguousarray(swarm["self"], dtype=np.int64)
            rc = lib().oracle_render_swarm_views(self.handle, ctypes.byref(make_params(p)), n,
                                                 _ptr(states, ctypes.c_double), _ptr(me, ctypes.c_int64),
                                                 allst.shape[0], _ptr(allst, ctypes.c_double), 1 if ub else 0,
                                                 _ptr(half, ctypes.c_double), _ptr(col, ctypes.c_uint8),
                                                 _ptr(depth, ctypes.c_double), _ptr(rgb, ctypes.c_uint8),
                                                 _ptr(hid, ctypes.c_int32), _ptr(tie, ctypes.c_uint8))
        else:
            half = np.ascontiguousarray(swarm["half"], dtype=np.float64)
            col = np.ascontiguousarray(swarm.get("rgb", (0, 0, 0)), dtype=np.uint8)
            rc = lib().oracle_render_swarm(self.handle, ctypes.byref(make_params(p)), n,
                                           _ptr(states, ctypes.c_double), 1 if ub else 0, _ptr(half, ctypes.c_double),
                                           _ptr(col, ctypes.c_uint8), _ptr(depth, ctypes.c_double),
                                           _ptr(rgb, ctypes.c_uint8), _ptr(hid, ctypes.c_int32),
                                           _ptr(tie, ctypes.c_uint8))
        if rc:
            raise ValueError(f"oracle_render failed ({rc})")
        return {"depth": depth, "rgb": rgb, "id": hid, "tie": tie.astype(bool)}

    def traversal_counts(self, p: dict, states: np.ndarray) -> dict:
        """Mean per ray, over every pixel of the agents' images, of the internal
        nodes and triangles a closest-hit walk of this scene's median-split BVH
        visits and tests (nearer child first).  A statistic, not a parity value."""
        if not self.bvh:
            raise ValueError("traversal counts need the oracle's BVH")
        states = _f64(states)
        out = np.zeros(2)
        rc = lib().oracle_traversal_counts(self.handle, ctypes.byref(make_params(p)), states.shape[0],
                                           _ptr(states, ctypes.c_double), _ptr(out, ctypes.c_double))
        if rc:
            raise ValueError(f"oracle_traversal_counts failed ({rc})")
        return {"nodes": float(out[0]), "tris": float(out[1])}

    def nearest(self, positions: np.ndarray, max_dist: float):
        """Closest mesh point of every query point: (dist [n], point [n,3], tri [n])."""
        pos = _f64(positions).reshape(-1, 3)
        n = pos.shape[0]
        dist = np.empty(n)
        point = np.empty((n, 3))
        tri = np.empty(n, np.int32)
        rc = lib().oracle_nearest(self.handle, n, _ptr(pos, ctypes.c_double), float(max_dist),
                                  _ptr(dist, ctypes.c_double), _ptr(point, ctypes.c_double),
                                  _ptr(tri, ctypes.c_int32))
        if rc:
            raise ValueError(f"oracle_nearest failed ({rc})")
        return dist, point, tri

    def point_triangle(self, positions: np.ndarray, ids: np.ndarray) -> np.ndarray:
        """Distance from each point to the given triangle (inf for an invalid id)."""
        pos = _f64(positions).reshape(-1, 3)
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        out = np.empty(pos.shape[0])
        lib().oracle_point_triangle(self.handle, pos.shape[0], _ptr(pos, ctypes.c_double),
                                    _ptr(ids, ctypes.c_int32), _ptr(out, ctypes.c_double))
        return out

    def validate(self, p: dict, states: np.ndarray, pix: np.ndarray, ids: np.ndarray, depth: np.ndarray,
                 swarm: dict | None = None):
        """Validity of claimed (id, depth) answers at flat pixel indices ``pix`` (see oracle.cpp)."""
        states = _f64(states)
        pix = np.ascontiguousarray(pix, dtype=np.int64)
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        depth = np.ascontiguousarray(depth, dtype=np.float32)
        valid = np.zeros(pix.shape[0], np.uint8)
        if swarm is None:
            rc = lib().oracle_validate(self.handle, ctypes.byref(make_params(p)), states.shape[0],
                                       _ptr(states, ctypes.c_double), pix.shape[0], _ptr(pix, ctypes.c_int64),
                                       _ptr(ids, ctypes.c_int32), _ptr(depth, ctypes.c_float),
                                       _ptr(valid, ctypes.c_uint8))
        elif "states" in swarm:
            half = np.ascontiguousarray(swarm["half"], dtype=np.float64)
            allst = _f64(swarm["states"])
            me = np.ascontiguousarray(swarm["self"], dtype=np.int64)
            rc = lib().oracle_validate_swarm_views(self.handle, ctypes.byref(make_params(p)), states.shape[0],
                                                   _ptr(states, ctypes.c_double), _ptr(me, ctypes.c_int64),
                                                   allst.shape[0], _ptr(allst, ctypes.c_double),
                                                   _ptr(half, ctypes.c_double), pix.shape[0],
                                                   _ptr(pix, ctypes.c_int64), _ptr(ids, ctypes.c_int32),
                                                   _ptr(depth, ctypes.c_float), _ptr(valid, ctypes.c_uint8))
        else:
            half = np.ascontiguousarray(swarm["half"], dtype=np.float64)
            rc = lib().oracle_validate_swarm(self.handle, ctypes.byref(make_params(p)), states.shape[0],
                                             _ptr(states, ctypes.c_double), _ptr(half, ctypes.c_double),
                                             pix.shape[0], _ptr(pix, ctypes.c_int64), _ptr(ids, ctypes.c_int32),
                                             _ptr(depth, ctypes.c_float), _ptr(valid, ctypes.c_uint8))
        if rc:
            raise ValueError(f"oracle_validate failed ({rc})")
        return valid.astype(bool)


def swarm_proximity(positions: np.ndarray, radius: float):
    """Brute-force pairwise proximity of one swarm (see oracle.cpp): per agent the
    nearest other agent's centre distance, its index and the number of others
    closer than 2 * radius."""
    pos = _f64(positions).reshape(-1, 3)
    n = pos.shape[0]
    dist = np.empty(n)
    other = np.empty(n, np.int32)
    hits = np.empty(n, np.int32)
    rc = lib().oracle_swarm_proximity(n, _ptr(pos, ctypes.c_double), float(radius), _ptr(dist, ctypes.c_double),
                                      _ptr(other, ctypes.c_int32), _ptr(hits, ctypes.c_int32))
    if rc:
        raise ValueError(f"oracle_swarm_proximity failed ({rc})")
    return dist, other, hits
