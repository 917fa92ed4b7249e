"""ctypes binding of libvisfly_b300.so (argument marshalling only).

Every function of ``include/visfly_b300.h`` is declared here with the same
name.  There is no fallback: if the shared library is missing or fails to
load, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvisfly_b300.so")
_lock = threading.Lock()
_lib = None

SIM_OK = 0
STATUS_NAMES = {0: "SIM_OK", -1: "SIM_ERR_INVALID_ARG", -2: "SIM_ERR_OOM", -3: "SIM_ERR_CUDA",
                -4: "SIM_ERR_NOT_FOUND", -5: "SIM_ERR_TRAVERSAL", -6: "SIM_ERR_TIMEOUT", -7: "SIM_ERR_BUDGET"}


class SimError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class SimParams(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_float), ("J", ctypes.c_float * 3), ("arm", ctypes.c_float), ("k", ctypes.c_float * 3),
        ("c_lag", ctypes.c_float), ("kappa", ctypes.c_float), ("rho", ctypes.c_float), ("Cd", ctypes.c_float * 3),
        ("area", ctypes.c_float * 3), ("omega_min", ctypes.c_float), ("omega_max", ctypes.c_float),
        ("a_max", ctypes.c_float), ("rate_max", ctypes.c_float * 3), ("K_rate", ctypes.c_float * 3),
        ("g", ctypes.c_float), ("dt", ctypes.c_float), ("n_sub", ctypes.c_int32), ("integrator", ctypes.c_int32),
        ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fov_deg", ctypes.c_float),
        ("max_depth", ctypes.c_float), ("cam_off", ctypes.c_float * 3), ("controller", ctypes.c_int32),
        ("K_pos", ctypes.c_float * 3), ("K_vel", ctypes.c_float * 3), ("K_att", ctypes.c_float * 3),
        ("K_omega", ctypes.c_float * 3),
    ]


class SceneInfo(ctypes.Structure):
    _fields_ = [("n_tris", ctypes.c_int64), ("n_nodes", ctypes.c_int64), ("n_large", ctypes.c_int64),
                ("depth", ctypes.c_int32), ("leaf_max", ctypes.c_int32), ("bytes", ctypes.c_int64)]


class RenderConfig(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("rays_per_lane", ctypes.c_int32),
                ("stack_in_smem", ctypes.c_int32), ("stack_depth", ctypes.c_int32),
                ("warps_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("stage_in_smem", ctypes.c_int32), ("node_width", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class RenderCounters(ctypes.Structure):
    _fields_ = [("node_visits", ctypes.c_int64), ("tri_tests", ctypes.c_int64), ("large_tests", ctypes.c_int64),
                ("items", ctypes.c_int64), ("rays", ctypes.c_int64), ("need_node_visits", ctypes.c_int64),
                ("need_tri_tests", ctypes.c_int64)]


class SimNoise(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("first_frame", ctypes.c_uint64), ("depth_gauss", ctypes.c_float),
                ("depth_speckle", ctypes.c_float), ("depth_shot", ctypes.c_float),
                ("depth_salt_pepper", ctypes.c_float), ("rgb_gauss", ctypes.c_float),
                ("rgb_speckle", ctypes.c_float), ("rgb_shot", ctypes.c_float), ("rgb_salt_pepper", ctypes.c_float),
                ("seg_dropout", ctypes.c_float), ("seg_gauss", ctypes.c_float), ("seg_speckle", ctypes.c_float),
                ("seg_shot", ctypes.c_float), ("seg_salt_pepper", ctypes.c_float), ("seg_max", ctypes.c_float)]


class SimSwarm(ctypes.Structure):
    _fields_ = [("half", ctypes.c_float * 3), ("rgb", ctypes.c_uint8 * 3), ("label", ctypes.c_int32)]


class SimRequest(ctypes.Structure):
    _fields_ = [("scene_id", ctypes.c_int32), ("n_agents", ctypes.c_int32), ("n_steps", ctypes.c_int32),
                ("frames", ctypes.c_int32), ("state0", ctypes.c_void_p), ("cmds", ctypes.c_void_p),
                ("state_out", ctypes.c_void_p), ("depth_out", ctypes.c_void_p), ("rgb_out", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("cancelled", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("iterations", ctypes.c_int64), ("agent_frames", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("active_requests", ctypes.c_int64), ("active_agents", ctypes.c_int64),
                ("mean_batch_agents", ctypes.c_double)]


def make_params(p: dict) -> SimParams:
    s = SimParams()
    for name, ctype in SimParams._fields_:
        v = p[name]
        if hasattr(ctype, "_length_"):
            setattr(s, name, ctype(*[float(x) for x in v]))
        elif ctype is ctypes.c_int32:
            setattr(s, name, int(v))
        else:
            setattr(s, name, float(v))
    return s


_vp, _i32, _i64, _sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
_P = ctypes.POINTER

SIGNATURES = {
    "sim_create_ctx": [_P(_vp), ctypes.c_int, _P(SimParams), _sz],
    "sim_destroy_ctx": [_vp],
    "sim_set_params": [_vp, _P(SimParams)],
    "sim_create_scene": [_vp, _vp, _i64, _vp, _i64, _vp, _P(_i32), _vp],
    "sim_destroy_scene": [_vp, _i32],
    "sim_scene_info_get": [_vp, _i32, _P(SceneInfo)],
    "sim_scene_build_times": [_vp, _i32, _P(ctypes.c_float), _P(ctypes.c_float)],
    "sim_step": [_vp, _i32, _vp, _vp, _vp, _vp],
    "sim_render": [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp],
    "sim_render_scene": [_vp, _i32, _i32, _vp, _vp, _vp, _vp, _vp],
    "sim_render_tile_costs": [_vp, _vp, _i64, _P(_i64)],
    "sim_kernel_timing": [_vp, _i32],
    "sim_kernel_times": [_vp, _vp, _i32, _P(_i32)],
    "sim_render_ex": [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "sim_scene_set_labels": [_vp, _i32, _vp, _i64],
    "sim_set_noise": [_vp, _vp],
    "sim_set_swarm": [_vp, _vp],
    "sim_env_create": [_vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp],
    "sim_env_run": [_vp, _vp, _vp],
    "sim_env_destroy": [_vp],
    "sim_swarm_proximity": [_vp, _i32, _vp, _vp, ctypes.c_float, _vp, _vp, _vp, _vp],
    "sim_render_scene_static": [_vp, _i32, _i32, _vp, _vp, _vp, _vp, _vp],
    "sim_step_backward": [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp],
    "sim_nearest_obstacle": [_vp, _i32, _vp, _vp, ctypes.c_float, _vp, _vp, _vp, _vp],
    "sim_rollout": [_vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp],
    "sim_rollout_backward": [_vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp],
    "sim_env_step": [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "sim_loop_create": [_vp, _P(_vp), _i32, _i32, _vp, _vp, _vp, _vp, _vp, _i32, _vp],
    "sim_loop_launch": [_vp, _vp],
    "sim_loop_destroy": [_vp],
    "sim_server_create": [_vp, _P(_vp), _i32],
    "sim_server_submit": [_vp, _P(SimRequest), _P(_i64)],
    "sim_server_wait": [_vp, _i64, _i32, _P(ctypes.c_double)],
    "sim_server_cancel": [_vp, _i64],
    "sim_server_stats_get": [_vp, _P(ServerStats)],
    "sim_server_destroy": [_vp],
    "sim_get_render_config": [_vp, _P(RenderConfig)],
    "sim_set_render_config": [_vp, _P(RenderConfig)],
    "sim_autotune_render": [_vp, _i32, _vp, _vp, _vp, _vp, _i32, _P(RenderConfig), _P(ctypes.c_float), _i32, _vp],
    "sim_render_config_list": [_P(RenderConfig), _i32],
    "sim_render_counted": [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _P(RenderCounters), _vp],
    "sim_get_status": [_vp, _vp, _i32],
    "sim_last_error": [_vp],
    "sim_mem_usage": [_vp, _P(_sz), _P(_sz)],
    "sim_probe_read_bandwidth": [_vp, _sz, _i32, _P(ctypes.c_double), _vp],
    "sim_version": [],
}
RESTYPES = {"sim_last_error": ctypes.c_char_p, "sim_version": ctypes.c_char_p}


def lib() -> ctypes.CDLL:
    """Load the in-tree shared library (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with python -m paper_2407_14783_b300.build")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = RESTYPES.get(name, ctypes.c_int)
            _lib = L
        return _lib


def check(code: int, where: str, ctx=None):
    if code != SIM_OK:
        msg = lib().sim_last_error(ctx).decode(errors="replace")
        raise SimError(code, where, msg)
