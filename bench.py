"""Benchmark of the rollout-step hot path on B300.

A step = one pass of the whole hot path over one batch: dynamics + controller
for every agent (sim_step) and the 64x64 depth + RGB render of every agent
(sim_render).  Default workload: one procedural cluttered room of 208,812
triangles (2,000 boxes / cylinders / icospheres in 50 x 50 x 6 m, about the
paper's 0.15 obstacles per cubic metre), 256 agents, RK4 at dt = 0.02,
hover-centred body-rate commands; agents are re-spawned (gym-style reset)
every 25 steps between timed steps.  Inputs are seeded and synthetic.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With torchrun (N > 1) every rank runs its own
agents in its own copy of the scene (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2407_14783_b300 import workloads as wl  # noqa: E402

METRIC = "agent-frames/s (dynamics+64x64 depth/RGB) on 1 B300"
EPISODE = 25
N_AGENTS = 256


def _hover(p):
    return math.sqrt(p["mass"] * p["g"] / 4.0 / p["k"][2]), 2.0 * p["g"] / p["a_max"] - 1.0


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.stop = threading.Event()
        self.t = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        while not self.stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                for line in out.stdout.strip().splitlines():
                    self.rows.append([x.strip() for x in line.split(",")])
            except Exception:
                pass
            self.stop.wait(0.2)

    def __enter__(self):
        self.t.start()
        return self

    def __exit__(self, *a):
        self.stop.set()
        self.t.join(timeout=10)

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for k, nm in enumerate(names):
                    if r[5 + k].lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_workload(rank: int):
    p = wl.params()
    scene = wl.cluttered_scene(seed=2)
    w_h, u_h = _hover(p)
    return p, scene, w_h, u_h


def run_reference(args):
    """The FP64 CPU oracle timed on the host cores on a bounded sample."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    p, scene, w_h, u_h = make_workload(0)
    osc = oracle.Scene.from_workload(scene)
    sample = 8
    spawn = wl.spawn_states(scene, sample, 3, w_h)
    cmds = wl.hover_commands(args.warmup + args.steps, sample, 4, u_h)
    s = spawn.copy()
    times = []
    for t in range(args.warmup + args.steps):
        if t % EPISODE == 0:
            s = spawn.copy()
        t0 = time.perf_counter()
        s = oracle.step(p, s, cmds[t])
        osc.render(p, s)
        dt = time.perf_counter() - t0
        if t >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = sample * len(times) / tot
    cores = oracle.num_threads()
    desc = f"{sample} of the 256 agents of the 208,812-triangle room per step, FP64 oracle (BVH traversal)"
    line = {"metric": METRIC, "value": value, "unit": "agent-frames/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "single large scene: 208,812 triangles, 256 agents, RK4 dt=0.02, 64x64 depth+RGB",
                       "sample_agents": sample},
            "cpu_baseline": {"value": value, "unit": "agent-frames/s", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "agent-frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_leg(p, scene, w_h, u_h, budget_s=15.0):
    """Oracle (as it stands) on a bounded sample of the same workload."""
    import oracle
    oracle.build()
    osc = oracle.Scene.from_workload(scene)
    sample = 8
    spawn = wl.spawn_states(scene, sample, 3, w_h)
    cmds = wl.hover_commands(1000, sample, 4, u_h)
    s = spawn.copy()
    n, t_used = 0, 0.0
    while t_used < budget_s and n < 1000:
        if n % EPISODE == 0:
            s = spawn.copy()
        t0 = time.perf_counter()
        s = oracle.step(p, s, cmds[n])
        osc.render(p, s)
        t_used += time.perf_counter() - t0
        n += 1
    return {"value": sample * n / t_used, "unit": "agent-frames/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{n} steps x {sample} agents of the 208,812-triangle room (dynamics + render, FP64)"}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2407_14783_b300.sim import Sim, to_soa

    ws, rank, local = _dist()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    p, scene, w_h, u_h = make_workload(rank)
    n = N_AGENTS
    K, W = args.steps, args.warmup
    sim = Sim(p, device=dev.index)
    sid = sim.add_workload_scene(scene)
    spawn = to_soa(wl.spawn_states(scene, n, 3 + 1000 * rank, w_h), dev)
    cmds = torch.tensor(np.ascontiguousarray(wl.hover_commands(W + K, n, 4 + 1000 * rank, u_h)
                                             .astype(np.float32).transpose(0, 2, 1)), device=dev)
    ids = torch.full((n,), sid, dtype=torch.int32, device=dev)
    state = spawn.clone()
    depth, rgb, _ = sim.alloc_images(n, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 126 MB L2
    stream = torch.cuda.current_stream()

    # warm-up (also selects the render configuration by autotuning on this workload)
    if args.no_autotune:
        best = sim.render_config()
    else:
        best, _ = sim.autotune(ids, state, depth, rgb, iters=3)
    for t in range(W):
        if t % EPISODE == 0:
            state.copy_(spawn)
        sim.step(state, cmds[t])
        sim.render(ids, state, depth, rgb)
    torch.cuda.synchronize()
    sim.check()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index if ws == 1 else local) as clk:
        for k in range(K):
            t = W + k
            if t % EPISODE == 0:
                state.copy_(spawn)
            flush.zero_()
            e0, e1, e2 = ev[k]
            e0.record(stream)
            sim.step(state, cmds[t])
            e1.record(stream)
            sim.render(ids, state, depth, rgb)
            e2.record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    sim.check()
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    dyn_ms = [a.elapsed_time(b) for a, b, c in ev]
    ren_ms = [b.elapsed_time(c) for a, b, c in ev]
    total_s = sum(step_ms) / 1e3
    if ws > 1:
        t = torch.tensor([total_s], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    value = ws * n * K / total_s

    # end to end through the public API with host buffers (pinned)
    cmd_host = cmds.cpu().pin_memory()
    depth_h = torch.empty((n, p["height"], p["width"]), dtype=torch.float32).pin_memory()
    rgb_h = torch.empty((n, p["height"], p["width"], 3), dtype=torch.uint8).pin_memory()
    K2 = min(K, 200)
    state.copy_(spawn)
    for t in range(3):
        sim.env_step(ids, state, cmd_host[t], depth_h, rgb_h)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(K2):
        if k % EPISODE == 0:
            state.copy_(spawn)
        sim.env_step(ids, state, cmd_host[W + k], depth_h, rgb_h)
        stream.synchronize()        # the host reads the observation every step
    e2e_s = time.perf_counter() - t0
    if ws > 1:
        t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": ws * n * K2 / e2e_s, "unit": "agent-frames/s", "h2d_bytes_per_step": 4 * 4 * n,
           "d2h_bytes_per_step": n * p["height"] * p["width"] * 7, "steps": K2}

    # traversal counters of one launch -> algorithmic bytes of the ray-cast kernel
    state.copy_(spawn)
    sim.step(state, cmds[W])
    cnt = sim.render(ids, state, depth, rgb, counted=True)
    items = max(cnt["items"], 1)
    rays_per_item = cnt["rays"] / items
    node_per_item = cnt["node_visits"] / items
    tri_per_item = (cnt["tri_tests"] + cnt["large_tests"]) / items
    fetched = cnt["node_visits"] * 64 + (cnt["tri_tests"] + cnt["large_tests"]) * 48
    out_bytes = n * p["height"] * p["width"] * 7 + n * 7 * 4
    render_ms = statistics.mean(ren_ms)
    hbm_peak, peak_kind = _peaks()
    achieved = (fetched + out_bytes) / (render_ms * 1e-3) / 1e9
    clocks = clk.summary()

    line = {"metric": METRIC, "value": value, "unit": "agent-frames/s", "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": 1e3 * total_s / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (procedural scene, seeded spawns and commands)",
            "config": {"workload": "single large scene: 208,812 triangles, 256 agents per GPU, RK4 dt=0.02, "
                                   "64x64 FP32 depth + uint8 RGB", "agents_per_gpu": n,
                       "triangles": int(scene.n_tris), "l2": "flushed between timed steps (256 MiB write)",
                       "reset_every_steps": EPISODE, "render_config": best},
            "e2e": e2e, "gpu_launches": 2 * K,
            "breakdown_ms": {"dynamics": statistics.mean(dyn_ms), "render": render_ms},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "raycast_kernel",
                         "bytes_per_launch": fetched + out_bytes,
                         "per_item": {"rays": rays_per_item, "node_fetches": node_per_item,
                                      "tri_fetches": tri_per_item}},
            "clocks": clocks}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_leg(p, scene, w_h, u_h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing leg")
    ap.add_argument("--no-autotune", action="store_true", help="use the default ray-cast configuration")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
