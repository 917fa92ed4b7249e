"""Continuous-batching step server (Python side of sim_server_*).

The server itself is native (a host thread inside libvisfly_b300.so); this
module only marshals requests.  A request advances n agents of one resident
scene by k steps with given commands and returns the final state and the
images of the last step (or of every step).
"""
from __future__ import annotations

import ctypes
import threading


from . import binding as B

FRAMES = {"none": 0, "last": 1, "all": 2}


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Server:
    def __init__(self, sim, capacity: int = 4096):
        self.sim = sim
        self.L = sim.L
        h = ctypes.c_void_p()
        B.check(self.L.sim_server_create(sim.h, ctypes.byref(h), capacity), "sim_server_create", sim.h)
        self.h = h
        self.capacity = capacity
        self._keep = {}
        self._lock = threading.Lock()

    def submit(self, scene: int, state0, cmds, state_out=None, depth_out=None, rgb_out=None,
               frames: str = "last") -> int:
        """state0 [17, n], cmds [T, 4, n] (host pinned or device, float32, contiguous);
        outputs as in sim_request.  Buffers are kept alive until wait() collects the ticket."""
        n = state0.shape[1]
        T = cmds.shape[0]
        for t, name in ((state0, "state0"), (cmds, "cmds"), (state_out, "state_out"), (depth_out, "depth_out"),
                        (rgb_out, "rgb_out")):
            if t is not None and not t.is_contiguous():
                raise ValueError(f"{name} must be contiguous")
        req = B.SimRequest(scene, n, T, FRAMES[frames], _p(state0), _p(cmds), _p(state_out), _p(depth_out),
                           _p(rgb_out))
        tk = ctypes.c_int64()
        B.check(self.L.sim_server_submit(self.h, ctypes.byref(req), ctypes.byref(tk)), "sim_server_submit",
                self.sim.h)
        with self._lock:
            self._keep[tk.value] = (state0, cmds, state_out, depth_out, rgb_out)
        return tk.value

    def wait(self, ticket: int, timeout_ms: int = -1) -> float:
        """Block until the request finishes; returns its latency in ms (raises on failure)."""
        lat = ctypes.c_double()
        rc = self.L.sim_server_wait(self.h, ticket, timeout_ms, ctypes.byref(lat))
        if rc != -6:  # SIM_ERR_TIMEOUT keeps the ticket alive
            with self._lock:
                self._keep.pop(ticket, None)
        B.check(rc, "sim_server_wait", self.sim.h)
        return lat.value

    def cancel(self, ticket: int):
        B.check(self.L.sim_server_cancel(self.h, ticket), "sim_server_cancel", self.sim.h)

    def stats(self) -> dict:
        st = B.ServerStats()
        B.check(self.L.sim_server_stats_get(self.h, ctypes.byref(st)), "sim_server_stats_get", self.sim.h)
        return {k: getattr(st, k) for k, _ in B.ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.sim_server_destroy(self.h)
            self.h = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
