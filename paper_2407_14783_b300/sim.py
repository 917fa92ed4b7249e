"""Python front end of the rollout-step library.

``Sim`` owns one library context on one GPU and forwards each call to the C ABI
(``binding``) with device pointers of torch tensors and the current CUDA
stream.  Tensors are plumbing only: every step of the path (dynamics, BVH
build, ray casting, adjoints) runs in the library's CUDA kernels.

Layouts follow the C header: state float32 [17, n] (structure of arrays),
commands float32 [4, n], images [n, H, W] / [n, H, W, 3].
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import binding as B

STATE_DIM = 17
CMD_DIM = 4


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


# The current stream's handle without building a torch.cuda.Stream object
# (3.3 us per call on the B300 host against 0.3 us); falls back to the public
# call where this torch has no such accessor.
_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream_handle(stream=None) -> int:
    if stream is not None:
        return stream.cuda_stream
    if _raw_stream is not None:
        return _raw_stream(torch.cuda.current_device())
    return torch.cuda.current_stream().cuda_stream


def _stream(stream=None):
    return ctypes.c_void_p(_stream_handle(stream))


def _need(t, dtype, shape, name):
    if t is None:
        return
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name}: need a contiguous CUDA {dtype} tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)} != {tuple(shape)}")


class Sim:
    """One simulation context: parameters, resident scenes and kernel settings."""

    def __init__(self, params: dict, device: int = 0, mem_budget: int = 0):
        self.L = B.lib()
        self.params = dict(params)
        self.device = device
        self.H, self.W = int(params["height"]), int(params["width"])
        h = ctypes.c_void_p()
        p = B.make_params(params)
        with torch.cuda.device(device):
            B.check(self.L.sim_create_ctx(ctypes.byref(h), device, ctypes.byref(p), mem_budget), "sim_create_ctx")
        self.h = h
        self.scenes = {}

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.sim_destroy_ctx(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------ set-up
    def set_params(self, params: dict):
        p = B.make_params(params)
        B.check(self.L.sim_set_params(self.h, ctypes.byref(p)), "sim_set_params", self.h)
        self.params = dict(params)
        self.H, self.W = int(params["height"]), int(params["width"])

    def add_scene(self, verts, tris, rgb, stream=None) -> int:
        v = np.ascontiguousarray(np.asarray(verts, np.float32))
        t = np.ascontiguousarray(np.asarray(tris, np.int32))
        c = np.ascontiguousarray(np.asarray(rgb, np.uint8))
        sid = ctypes.c_int32(-1)
        rc = self.L.sim_create_scene(self.h, v.ctypes.data, v.shape[0], t.ctypes.data, t.shape[0], c.ctypes.data,
                                     ctypes.byref(sid), _stream(stream))
        B.check(rc, "sim_create_scene", self.h)
        self.scenes[sid.value] = t.shape[0]
        return sid.value

    def add_workload_scene(self, scene, stream=None) -> int:
        return self.add_scene(scene.verts, scene.tris, scene.rgb, stream)

    def remove_scene(self, sid: int):
        B.check(self.L.sim_destroy_scene(self.h, sid), "sim_destroy_scene", self.h)
        self.scenes.pop(sid, None)

    def scene_info(self, sid: int) -> dict:
        info = B.SceneInfo()
        B.check(self.L.sim_scene_info_get(self.h, sid, ctypes.byref(info)), "sim_scene_info_get", self.h)
        return {k: int(getattr(info, k)) for k, _ in B.SceneInfo._fields_}

    BUILD_PHASES = ("bounds", "morton", "sort", "radix_tree", "refit", "clustering", "tree_pack", "tri_pack")

    def scene_build_times(self, sid: int) -> dict:
        """Milliseconds per build phase of scene sid, and the whole call's host time."""
        ms = (ctypes.c_float * len(self.BUILD_PHASES))()
        wall = ctypes.c_float()
        B.check(self.L.sim_scene_build_times(self.h, sid, ms, ctypes.byref(wall)), "sim_scene_build_times", self.h)
        out = {k: float(v) for k, v in zip(self.BUILD_PHASES, ms)}
        out["wall"] = float(wall.value)
        return out

    # ------------------------------------------------------------ dynamics
    def step(self, state, cmd, ckpt=None, stream=None):
        n = state.shape[1]
        _need(state, torch.float32, (STATE_DIM, n), "state")
        _need(cmd, torch.float32, (CMD_DIM, n), "cmd")
        _need(ckpt, torch.float32, (STATE_DIM, n), "ckpt")
        B.check(self.L.sim_step(self.h, n, _ptr(state), _ptr(cmd), _ptr(ckpt), _stream(stream)), "sim_step", self.h)
        return state

    def step_backward(self, state_in, cmd, g_state_out, stream=None):
        n = state_in.shape[1]
        _need(state_in, torch.float32, (STATE_DIM, n), "state_in")
        _need(cmd, torch.float32, (CMD_DIM, n), "cmd")
        _need(g_state_out, torch.float32, (STATE_DIM, n), "g_state_out")
        g_in = torch.empty_like(state_in)
        g_cmd = torch.empty_like(cmd)
        rc = self.L.sim_step_backward(self.h, n, _ptr(state_in), _ptr(cmd), _ptr(g_state_out), _ptr(g_in),
                                      _ptr(g_cmd), _stream(stream))
        B.check(rc, "sim_step_backward", self.h)
        return g_in, g_cmd

    def rollout(self, state0, cmds, K: int = 10, keep_states: bool = True, stream=None):
        """T steps in one launch.  Returns (states [T+1,17,n] or None, ckpt [ceil(T/K),17,n], final [17,n])."""
        T, n = cmds.shape[0], state0.shape[1]
        _need(state0, torch.float32, (STATE_DIM, n), "state0")
        _need(cmds, torch.float32, (T, CMD_DIM, n), "cmds")
        dev = state0.device
        states = torch.empty((T + 1, STATE_DIM, n), device=dev) if keep_states else None
        nck = (T + K - 1) // K
        ckpt = torch.empty((max(nck, 1), STATE_DIM, n), device=dev)
        final = torch.empty((STATE_DIM, n), device=dev)
        rc = self.L.sim_rollout(self.h, n, T, K, _ptr(state0), _ptr(cmds), _ptr(states), _ptr(ckpt), _ptr(final),
                                _stream(stream))
        B.check(rc, "sim_rollout", self.h)
        return states, ckpt, final

    def rollout_backward(self, ckpt, cmds, g_states, K: int = 10, stream=None):
        T, n = cmds.shape[0], cmds.shape[2]
        _need(cmds, torch.float32, (T, CMD_DIM, n), "cmds")
        _need(g_states, torch.float32, (T + 1, STATE_DIM, n), "g_states")
        g0 = torch.empty((STATE_DIM, n), device=cmds.device)
        gc = torch.empty_like(cmds)
        rc = self.L.sim_rollout_backward(self.h, n, T, K, _ptr(ckpt), _ptr(cmds), _ptr(g_states), _ptr(g0),
                                         _ptr(gc), _stream(stream))
        B.check(rc, "sim_rollout_backward", self.h)
        return g0, gc

    # ------------------------------------------------------------ rendering
    def alloc_images(self, n: int, depth=True, rgb=True, hit=False, device=None):
        dev = device if device is not None else torch.device("cuda", self.device)
        d = torch.empty((n, self.H, self.W), device=dev) if depth else None
        c = torch.empty((n, self.H, self.W, 3), dtype=torch.uint8, device=dev) if rgb else None
        i = torch.empty((n, self.H, self.W), dtype=torch.int32, device=dev) if hit else None
        return d, c, i

    def render(self, scene_of_agent, state, depth=None, rgb=None, hit=None, stream=None, counted=False):
        n = state.shape[1]
        _need(scene_of_agent, torch.int32, (n,), "scene_of_agent")
        _need(state, torch.float32, (STATE_DIM, n), "state")
        _need(depth, torch.float32, (n, self.H, self.W), "depth")
        _need(rgb, torch.uint8, (n, self.H, self.W, 3), "rgb")
        _need(hit, torch.int32, (n, self.H, self.W), "hit")
        if counted:
            cnt = B.RenderCounters()
            rc = self.L.sim_render_counted(self.h, n, _ptr(scene_of_agent), _ptr(state), _ptr(depth), _ptr(rgb),
                                           _ptr(hit), ctypes.byref(cnt), _stream(stream))
            B.check(rc, "sim_render_counted", self.h)
            return {k: int(getattr(cnt, k)) for k, _ in B.RenderCounters._fields_}
        rc = self.L.sim_render(self.h, n, _ptr(scene_of_agent), _ptr(state), _ptr(depth), _ptr(rgb), _ptr(hit),
                               _stream(stream))
        B.check(rc, "sim_render", self.h)
        return depth, rgb, hit

    def tile_costs(self) -> np.ndarray:
        """Traversal cost of every tile of the last sim_render launch:
        uint32 [n, tiles_y, tiles_x] (see sim_render_tile_costs)."""
        k = ctypes.c_int64()
        B.check(self.L.sim_render_tile_costs(self.h, None, 0, ctypes.byref(k)), "sim_render_tile_costs", self.h)
        out = np.zeros(k.value, np.uint32)
        B.check(self.L.sim_render_tile_costs(self.h, out.ctypes.data_as(ctypes.c_void_p), k.value, ctypes.byref(k)),
                "sim_render_tile_costs", self.h)
        cfg = self.render_config()
        tx, ty = -(-self.W // cfg["tile_w"]), -(-self.H // cfg["tile_h"])
        return out.reshape(-1, ty, tx)

    KERNEL_TIMING_MAX = 1024

    def kernel_timing(self, enable: bool = True):
        """Record the device time of each following ray-cast launch alone (CUDA
        events around the kernel; see sim_kernel_timing); clears the record."""
        B.check(self.L.sim_kernel_timing(self.h, 1 if enable else 0), "sim_kernel_timing", self.h)

    def kernel_times(self) -> np.ndarray:
        """Milliseconds of each ray-cast launch recorded since timing was turned
        on (at most KERNEL_TIMING_MAX), in launch order; clears the record."""
        out = np.zeros(self.KERNEL_TIMING_MAX, np.float32)
        k = ctypes.c_int32()
        B.check(self.L.sim_kernel_times(self.h, out.ctypes.data_as(ctypes.c_void_p), len(out), ctypes.byref(k)),
                "sim_kernel_times", self.h)
        return out[:min(k.value, len(out))].copy()

    def nearest_obstacle(self, scene_of_agent, state, max_dist: float = 10.0, stream=None):
        """Closest mesh point of every agent: (dist [n], point [3, n], tri [n])."""
        n = state.shape[1]
        _need(scene_of_agent, torch.int32, (n,), "scene_of_agent")
        _need(state, torch.float32, (STATE_DIM, n), "state")
        dist = torch.empty((n,), device=state.device)
        point = torch.empty((3, n), device=state.device)
        tri = torch.empty((n,), dtype=torch.int32, device=state.device)
        rc = self.L.sim_nearest_obstacle(self.h, n, _ptr(scene_of_agent), _ptr(state), float(max_dist), _ptr(dist),
                                         _ptr(point), _ptr(tri), _stream(stream))
        B.check(rc, "sim_nearest_obstacle", self.h)
        return dist, point, tri

    def set_swarm(self, half=None, rgb=(255, 255, 255), label: int = -2):
        """Multi-agent mode: agents sharing a scene see each other's drones, boxes
        of half extents `half` (m); None returns to the parallel-agents mode."""
        if half is None:
            B.check(self.L.sim_set_swarm(self.h, None), "sim_set_swarm", self.h)
            return
        cfg = B.SimSwarm((ctypes.c_float * 3)(*[float(x) for x in half]), (ctypes.c_uint8 * 3)(*[int(x) for x in rgb]),
                         int(label))
        B.check(self.L.sim_set_swarm(self.h, ctypes.byref(cfg)), "sim_set_swarm", self.h)

    def swarm_proximity(self, scene_of_agent, state, radius: float, stream=None):
        """Per agent, over the other agents of its scene: (nearest centre distance,
        that agent, number closer than 2 radius)."""
        n = state.shape[1]
        _need(scene_of_agent, torch.int32, (n,), "scene_of_agent")
        _need(state, torch.float32, (STATE_DIM, n), "state")
        dist = torch.empty((n,), device=state.device)
        other = torch.empty((n,), dtype=torch.int32, device=state.device)
        hits = torch.empty((n,), dtype=torch.int32, device=state.device)
        rc = self.L.sim_swarm_proximity(self.h, n, _ptr(scene_of_agent), _ptr(state), float(radius), _ptr(dist),
                                        _ptr(other), _ptr(hits), _stream(stream))
        B.check(rc, "sim_swarm_proximity", self.h)
        return dist, other, hits

    def render_seg(self, scene_of_agent, state, depth=None, rgb=None, hit=None, seg=None, stream=None):
        """Render with a segmentation image (labels of sim_scene_set_labels, -1 on a miss)."""
        n = state.shape[1]
        _need(scene_of_agent, torch.int32, (n,), "scene_of_agent")
        _need(state, torch.float32, (STATE_DIM, n), "state")
        _need(depth, torch.float32, (n, self.H, self.W), "depth")
        _need(rgb, torch.uint8, (n, self.H, self.W, 3), "rgb")
        _need(hit, torch.int32, (n, self.H, self.W), "hit")
        _need(seg, torch.int32, (n, self.H, self.W), "seg")
        rc = self.L.sim_render_ex(self.h, n, _ptr(scene_of_agent), _ptr(state), _ptr(depth), _ptr(rgb), _ptr(hit),
                                  _ptr(seg), _stream(stream))
        B.check(rc, "sim_render_ex", self.h)
        return depth, rgb, hit, seg

    def set_labels(self, sid: int, labels):
        lab = np.ascontiguousarray(np.asarray(labels, np.int32))
        B.check(self.L.sim_scene_set_labels(self.h, sid, lab.ctypes.data, lab.shape[0]), "sim_scene_set_labels",
                self.h)

    def set_noise(self, cfg: dict | None):
        """cfg keys as in sim_noise (missing ones 0); None for clean images."""
        if cfg is None:
            B.check(self.L.sim_set_noise(self.h, None), "sim_set_noise", self.h)
            return
        nz = B.SimNoise(**{k: cfg.get(k, 0) for k, _ in B.SimNoise._fields_})
        B.check(self.L.sim_set_noise(self.h, ctypes.byref(nz)), "sim_set_noise", self.h)

    def render_config(self) -> dict:
        c = B.RenderConfig()
        B.check(self.L.sim_get_render_config(self.h, ctypes.byref(c)), "sim_get_render_config", self.h)
        return c.as_dict()

    def set_render_config(self, cfg: dict):
        c = B.RenderConfig(**{k: int(v) for k, v in cfg.items()})
        B.check(self.L.sim_set_render_config(self.h, ctypes.byref(c)), "sim_set_render_config", self.h)

    @staticmethod
    def render_configs() -> list:
        L = B.lib()
        n = L.sim_render_config_list(None, 0)
        arr = (B.RenderConfig * n)()
        L.sim_render_config_list(arr, n)
        return [a.as_dict() for a in arr]

    def autotune(self, scene_of_agent, state, depth, rgb, iters: int = 5, stream=None):
        n = state.shape[1]
        best = B.RenderConfig()
        nc = len(self.render_configs())
        times = (ctypes.c_float * nc)(*([float("nan")] * nc))
        rc = self.L.sim_autotune_render(self.h, n, _ptr(scene_of_agent), _ptr(state), _ptr(depth), _ptr(rgb), iters,
                                        ctypes.byref(best), times, nc, _stream(stream))
        B.check(rc, "sim_autotune_render", self.h)
        return best.as_dict(), list(times)

    def make_loop(self, scene_of_agent, state, cmds, depth=None, rgb=None, stream=None) -> "Loop":
        """Capture len(cmds) steps (step + render) into one CUDA graph.  depth / rgb
        hold F frame slots ([F, n, H, W] / [F, n, H, W, 3]); step t writes slot t % F."""
        T, n = cmds.shape[0], state.shape[1]
        _need(scene_of_agent, torch.int32, (n,), "scene_of_agent")
        _need(state, torch.float32, (STATE_DIM, n), "state")
        _need(cmds, torch.float32, (T, CMD_DIM, n), "cmds")
        F = depth.shape[0] if depth is not None else (rgb.shape[0] if rgb is not None else 1)
        _need(depth, torch.float32, (F, n, self.H, self.W), "depth")
        _need(rgb, torch.uint8, (F, n, self.H, self.W, 3), "rgb")
        h = ctypes.c_void_p()
        rc = self.L.sim_loop_create(self.h, ctypes.byref(h), n, T, _ptr(scene_of_agent), _ptr(state), _ptr(cmds),
                                    _ptr(depth), _ptr(rgb), F, _stream(stream))
        B.check(rc, "sim_loop_create", self.h)
        return Loop(self, h, (scene_of_agent, state, cmds, depth, rgb))

    # ------------------------------------------------------------ env step with host buffers
    def env_step(self, scene_of_agent, state, cmd_host, depth_host=None, rgb_host=None, state_host=None,
                 stream=None):
        """One environment step with host buffers (see sim_env_step): host
        commands in, host images (and optionally the state) out.  Called once
        per control step, so the marshalling stays minimal: raw pointers, no
        per-call ctypes objects."""
        n = state.shape[1]
        ptr = [None, None, None, None]
        for i, t in enumerate((cmd_host, depth_host, rgb_host, state_host)):
            if t is not None:
                if t.is_cuda or not t.is_contiguous():
                    raise ValueError(f"{('cmd_host', 'depth_host', 'rgb_host', 'state_host')[i]}: "
                                     "need a contiguous host tensor")
                ptr[i] = t.data_ptr()
        s = _stream_handle(stream)
        rc = self.L.sim_env_step(self.h, n, scene_of_agent.data_ptr(), state.data_ptr(), ptr[0], ptr[1], ptr[2],
                                 ptr[3], s)
        if rc:
            B.check(rc, "sim_env_step", self.h)

    def make_env(self, scene_of_agent, state, depth_host=None, rgb_host=None, state_host=None) -> "Env":
        """A prepared environment step over fixed agents and page-locked host
        buffers (see sim_env_create): Env.step(cmd_host) runs one step."""
        n = state.shape[1]
        _need(scene_of_agent, torch.int32, (n,), "scene_of_agent")
        _need(state, torch.float32, (STATE_DIM, n), "state")
        for t, name, shape in ((depth_host, "depth_host", (n, self.H, self.W)),
                               (rgb_host, "rgb_host", (n, self.H, self.W, 3)), (state_host, "state_host", (STATE_DIM, n))):
            if t is not None and (t.is_cuda or not t.is_contiguous() or tuple(t.shape) != shape):
                raise ValueError(f"{name}: need a contiguous host tensor of shape {shape}")
        h = ctypes.c_void_p()
        rc = self.L.sim_env_create(self.h, ctypes.byref(h), n, _ptr(scene_of_agent), _ptr(state), _ptr(depth_host),
                                   _ptr(rgb_host), _ptr(state_host))
        B.check(rc, "sim_env_create", self.h)
        return Env(self, h, n, (scene_of_agent, state, depth_host, rgb_host, state_host))

    # ------------------------------------------------------------ status
    def status(self, timeout_ms: int = 10000, stream=None) -> int:
        return int(self.L.sim_get_status(self.h, _stream(stream), timeout_ms))

    def check(self, timeout_ms: int = 10000, stream=None):
        B.check(self.L.sim_get_status(self.h, _stream(stream), timeout_ms), "sim_get_status", self.h)

    def mem_usage(self):
        u, b = ctypes.c_size_t(), ctypes.c_size_t()
        self.L.sim_mem_usage(self.h, ctypes.byref(u), ctypes.byref(b))
        return u.value, b.value

    def probe_read_bandwidth(self, nbytes: int, iters: int = 20, stream=None) -> float:
        g = ctypes.c_double()
        B.check(self.L.sim_probe_read_bandwidth(self.h, nbytes, iters, ctypes.byref(g), _stream(stream)),
                "sim_probe_read_bandwidth", self.h)
        return g.value


class Env:
    """A prepared environment step (see Sim.make_env); keeps its buffers alive."""

    def __init__(self, sim, h, n, keep):
        self.sim, self.h, self.n, self._keep = sim, h, n, keep
        self._run = sim.L.sim_env_run

    def step(self, cmd_host, stream=None):
        """One environment step with host commands float32 [4, n]."""
        if cmd_host.is_cuda or not cmd_host.is_contiguous() or cmd_host.numel() != 4 * self.n:
            raise ValueError("cmd_host: need a contiguous host tensor of 4 * n floats")
        s = _stream_handle(stream)
        rc = self._run(self.h, cmd_host.data_ptr(), s)
        if rc:
            B.check(rc, "sim_env_run", self.sim.h)

    def close(self):
        if self.h and self.h.value:
            self.sim.L.sim_env_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Loop:
    """A captured step loop (see Sim.make_loop); keeps its buffers alive."""

    def __init__(self, sim, h, keep):
        self.sim, self.h, self._keep = sim, h, keep

    def launch(self, stream=None):
        B.check(self.sim.L.sim_loop_launch(self.h, _stream(stream)), "sim_loop_launch", self.sim.h)

    def close(self):
        if self.h and self.h.value:
            self.sim.L.sim_loop_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Rollout(torch.autograd.Function):
    """Differentiable T-step rollout through the library's kernels.

    forward(sim, state0 [17,n], cmds [T,4,n], K) -> states [T+1,17,n]
    The forward keeps only checkpoints every K steps; backward re-runs each
    K-step segment from its checkpoint on the GPU and sweeps it backwards with
    the hand-written adjoint.
    """

    @staticmethod
    def forward(ctx, sim, state0, cmds, K=10):
        states, ckpt, _ = sim.rollout(state0.contiguous(), cmds.contiguous(), K=K, keep_states=True)
        ctx.sim, ctx.K = sim, K
        ctx.save_for_backward(ckpt, cmds)
        return states

    @staticmethod
    def backward(ctx, g_states):
        ckpt, cmds = ctx.saved_tensors
        g0, gc = ctx.sim.rollout_backward(ckpt, cmds.contiguous(), g_states.contiguous(), K=ctx.K)
        return None, g0, gc, None


def rollout(sim: Sim, state0, cmds, K: int = 10):
    return Rollout.apply(sim, state0, cmds, K)


def to_soa(x: np.ndarray, device="cuda") -> torch.Tensor:
    """[n, d] host array -> contiguous float32 [d, n] device tensor."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.float32).T)).to(device)


def from_soa(t: torch.Tensor) -> np.ndarray:
    """[d, n] device tensor -> [n, d] float64 host array."""
    return t.detach().cpu().numpy().T.astype(np.float64)
