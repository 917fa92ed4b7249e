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
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2407_14783_b300 import workloads as wl  # noqa: E402

METRIC = "agent-frames/s (dynamics+64x64 depth/RGB) on 1 B300"
BATCHED_LOOPS = 3                 # timed 100-step graph launches of the batched leg
SERVE_LOAD, SERVE_SECONDS = 0.5, 2.0  # the serving leg: half the offered load, 2 s of arrivals
BUILD_SCENE = (2_000_000, 901)    # (triangles, seed) of the scene whose build phases are timed
EPISODE = 25
E2E_WARMUP_S = 0.5
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
    """nvidia-smi clocks and throttle reasons sampled every 20 ms during the
    timed region (one nvidia-smi process in loop mode)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)  # first sample lands before the timed region starts
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is None:
            return
        time.sleep(0.05)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.strip().splitlines():
            self.rows.append([x.strip() for x in line.split(",")])

    def summary(self):
        ok = [r for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        sm = [float(r[1]) for r in ok]
        mx = [float(r[2]) for r in ok if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in ok:
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
    # warm-up: the W untimed steps and at least E2E_WARMUP_S seconds of steps,
    # so that the host cores run at their settled rate when timing starts
    s = spawn.copy()
    t_w, k = time.perf_counter(), 0
    while k < args.warmup or time.perf_counter() - t_w < E2E_WARMUP_S:
        if k % EPISODE == 0:
            s = spawn.copy()
        s = oracle.step(p, s, cmds[k % len(cmds)])
        osc.render(p, s)
        k += 1
    s = spawn.copy()
    times = []
    for t in range(args.warmup, args.warmup + args.steps):
        if t % EPISODE == 0:
            s = spawn.copy()
        t0 = time.perf_counter()
        s = oracle.step(p, s, cmds[t])
        osc.render(p, s)
        times.append(time.perf_counter() - t0)
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


def cpu_baseline_leg(p, scene, w_h, u_h, count_states=None, budget_s=15.0):
    """Oracle (as it stands) on a bounded sample of the same workload.  With
    count_states ([n, 17], the poses of the GPU's counted launch) it also walks
    the oracle's own median-split BVH for every ray of those images and reports
    the mean internal nodes and triangles per ray beside the GPU's counts."""
    import oracle
    oracle.build()
    osc = oracle.Scene.from_workload(scene)
    walk = None
    if count_states is not None:
        walk = osc.traversal_counts(p, count_states)
        walk["rays"] = int(count_states.shape[0] * p["width"] * p["height"])
        walk["what"] = ("closest-hit walks, nearer child first, of the oracle's median-split BVH (leaves of up to "
                        "4 triangles, large triangles inside the tree): mean internal nodes visited and "
                        "triangles tested per ray")
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
    # the tiny configuration in full (4 agents, 10 steps, 492 triangles), by
    # brute force and by the oracle's own BVH
    tiny = wl.room_scene()
    st0 = wl.spawn_states(tiny, 4, 11, w_h)
    tc = wl.uniform_commands(10, 4, 12)
    tiny_s = {}
    for mode, bvh in (("brute_force", False), ("bvh", True)):
        ot = oracle.Scene.from_workload(tiny, bvh=bvh)
        st = st0.copy()
        t0 = time.perf_counter()
        for k in range(10):
            st = oracle.step(p, st, tc[k])
            ot.render(p, st, use_bvh=bvh)
        tiny_s[mode] = 40 / (time.perf_counter() - t0)
    return {"value": sample * n / t_used, "unit": "agent-frames/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{n} steps x {sample} agents of the 208,812-triangle room (dynamics + render, FP64)",
            "tiny_config_agent_frames_per_s": tiny_s, "oracle_bvh_per_ray": walk}


def _recorded_profile():
    """Figures of one ray-cast launch from the committed ncu summary, if it was
    taken on the current kernel source (matching SHA-1), else {}: DRAM bytes per
    launch and the issue-active and ALU-pipe fractions."""
    import hashlib
    src = os.path.join(ROOT, "paper_2407_14783_b300", "csrc", "raycast.cu")
    prof = os.path.join(ROOT, "profiles", "raycast_large_scene_256agents.md")
    try:
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
        for line in open(prof):
            if line.startswith("dram_bytes_per_launch"):
                parts = dict((k.strip(), v.strip()) for k, v in
                             (kv.split("=", 1) for kv in line.split(";") if "=" in kv))
                if parts.get("raycast_cu_sha1", "") == sha:
                    out = {"traffic": int(parts["dram_bytes_per_launch"])}
                    for k in parts:
                        if k in ("issue_active", "alu_pipe", "l2_throughput", "dram_throughput") or \
                                k.startswith("warp_inst_per_launch"):
                            out[k] = float(parts[k])
                    return out
    except Exception:
        pass
    return {}


# Table II sensor noise at the strengths the sensor parity test uses: depth,
# colour and segmentation each with Gaussian, speckle, Poisson and
# salt-and-pepper noise, plus label dropout.
SENSOR_NOISE = {"seed": 1234, "first_frame": 5, "depth_gauss": 0.02, "depth_speckle": 0.01, "depth_shot": 50.0,
                "depth_salt_pepper": 0.01, "rgb_gauss": 3.0, "rgb_speckle": 0.02, "rgb_shot": 0.5,
                "rgb_salt_pepper": 0.01, "seg_dropout": 0.05, "seg_gauss": 0.8, "seg_speckle": 0.01, "seg_shot": 2.0,
                "seg_salt_pepper": 0.02, "seg_max": 60}


def _event_ms(fn, flush, reps):
    """Mean CUDA-event time of fn() on the current stream, the L2 flushed before each call."""
    import torch
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        ts.append((e0, e1))
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in ts)


def sensor_extra(sim, scene, sid, ids, state, depth, rgb, flush, n, p, reps=30):
    """The sensor epilogue (Sec. III-B, Table II): the same renders with a
    segmentation image, then with every noise model on."""
    import torch
    sim.set_labels(sid, np.arange(scene.n_tris, dtype=np.int32) % 60)
    seg = torch.empty((n, p["height"], p["width"]), dtype=torch.int32, device=state.device)
    plain = _event_ms(lambda: sim.render(ids, state, depth, rgb), flush, reps)
    with_seg = _event_ms(lambda: sim.render_seg(ids, state, depth, rgb, None, seg), flush, reps)
    sim.set_noise(SENSOR_NOISE)
    noisy = _event_ms(lambda: sim.render_seg(ids, state, depth, rgb, None, seg), flush, reps)
    # a lighter setting: additive Gaussian noise on depth and colour only
    sim.set_noise({"seed": 1234, "depth_gauss": 0.02, "rgb_gauss": 3.0})
    gauss = _event_ms(lambda: sim.render(ids, state, depth, rgb), flush, reps)
    sim.set_noise(None)
    sim.check()
    return {"agents": n, "render_ms": plain, "with_segmentation_ms": with_seg, "with_segmentation_and_noise_ms": noisy,
            "with_depth_and_rgb_gauss_ms": gauss, "agent_frames_per_s_all_sensors": n / (noisy * 1e-3),
            "pose": "fixed (spawn + one step)"}


def controller_extra(sim, p, spawn, n, u_h):
    """Device time of one control step per controller and integrator setting,
    20 steps captured in a CUDA graph (no launch gaps)."""
    import torch
    dev = spawn.device
    rng = np.random.default_rng(5)
    hover = torch.tensor(np.ascontiguousarray(np.broadcast_to([[u_h], [0.0], [0.0], [0.0]], (4, n)), dtype=np.float32),
                         device=dev)
    u_srt = 2.0 * p["mass"] * p["g"] / 4 / (p["k"][2] * p["omega_max"] ** 2) - 1.0
    srt = torch.full((4, n), u_srt, dtype=torch.float32, device=dev)
    vel = torch.tensor(np.vstack([rng.uniform(-1, 1, (3, n)), np.zeros((1, n))]).astype(np.float32), device=dev)
    pos = spawn[0:4].clone()
    pos[0:3] += torch.tensor(rng.uniform(-1.5, 1.5, (3, n)).astype(np.float32), device=dev)
    pos[3] = 0.0
    cases = (("ctbr_rk4", {}, hover), ("ctbr_euler", {"integrator": 1}, hover), ("ctbr_rk4_4_substeps", {"n_sub": 4}, hover),
             ("srt_rk4", {"controller": 1}, srt), ("lv_rk4", {"controller": 2}, vel), ("ps_rk4", {"controller": 3}, pos))
    out = {}
    for name, over, cmd in cases:
        sim.set_params({**p, **over})
        st = spawn.clone()
        for _ in range(3):
            sim.step(st, cmd)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(20):
                sim.step(st, cmd)
        graph.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) / 20 * 1e3
        del graph
        out[name] = {"us_per_step": us, "agent_steps_per_s": n / (us * 1e-6)}
    sim.set_params(p)
    sim.check()
    out["agents"] = n
    return out


def raycast_roofline(sim, cnt, n, p, launch_ms, sm_mhz=None, cfg=None):
    """Roofline of the dominant kernel.  Algorithmic bytes per launch (per agent-frame:
    4096 rays x (N_node * 64 B + N_tri * 48 B + 7 B output) + 28 B of pose), with
    N_node / N_tri the nodes and triangles each ray's own walk needs (counter build),
    over the ray-cast kernel's average launch time, against this GPU's L2 read bandwidth measured by
    the library's probe (the scene is L2-resident)."""
    rays = cnt["rays"]
    items = max(cnt["items"], 1)
    rays_per_item = rays / items
    need_nodes = cnt["need_node_visits"] / rays
    need_tris = (cnt["need_tri_tests"] + cnt["large_tests"] * rays_per_item) / rays
    per_ray = need_nodes * 64 + need_tris * 48 + 7
    alg_bytes = rays * per_ray + n * 28
    achieved = alg_bytes / (launch_ms * 1e-3) / 1e9
    # the peak is the best of five probe runs (single runs vary by several per cent)
    l2 = max(sim.probe_read_bandwidth(64 << 20, iters=20) for _ in range(5))
    hbm, hbm_kind = _peaks()
    prof = _recorded_profile()
    traffic = prof.get("traffic")
    hbm_achieved = traffic / (launch_ms * 1e-3) / 1e9 if traffic else None
    return {"bound": "l2", "achieved": achieved, "peak": l2, "unit": "GB/s", "frac": achieved / l2,
            "traffic": traffic, "kernel": "raycast_kernel",
            "hbm_achieved": hbm_achieved, "hbm_frac": hbm_achieved / hbm if hbm_achieved else None,
            "peak_kind": "L2 read bandwidth measured in this run (sim_probe_read_bandwidth, 64 MiB resident, "
                         "best of 5)",
            "hbm_peak": hbm, "hbm_peak_kind": hbm_kind, "alg_bytes_per_launch": alg_bytes,
            "launch_ms": launch_ms,
            "per_ray": {"need_nodes": need_nodes, "need_tris": need_tris, "bytes": per_ray},
            "per_item": {"rays": rays_per_item, "node_fetches": cnt["node_visits"] / items,
                         "tri_fetches": cnt["tri_tests"] / items, "large_tests": cnt["large_tests"] / items},
            "packet_demand_gbs": (cnt["node_visits"] * 64 + (cnt["tri_tests"] + cnt["large_tests"]) * 48)
                                 * rays_per_item / (launch_ms * 1e-3) / 1e9,
            # what limits the kernel in the committed ncu capture of this source:
            # instruction issue, not L2 or DRAM bandwidth
            "ncu": {k: prof[k] for k in ("issue_active", "alu_pipe", "l2_throughput", "dram_throughput")
                    if k in prof} or None,
            "issue": issue_roofline(prof, launch_ms, sm_mhz, cfg)}


def issue_roofline(prof, launch_ms, sm_mhz, cfg=None):
    """The bound the ray cast actually meets: instruction issue.  Warp
    instructions of one launch (the committed ncu capture of this source, same
    workload, the timed configuration's tile shape where the capture has it)
    over the launch's CUDA-event time, against the SMs' issue peak of one warp
    instruction per cycle per scheduler (the device's SMs x 4 schedulers x the
    SM clock sampled during the timed steps)."""
    import torch
    shape = "%dx%d" % (cfg["tile_w"], cfg["tile_h"]) if cfg else None
    inst = prof.get("warp_inst_per_launch_" + shape) if shape else None
    source = shape if inst else "8x4"
    inst = inst or prof.get("warp_inst_per_launch")
    if not inst or not sm_mhz:
        return None
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    achieved = inst / (launch_ms * 1e-3) / 1e9
    peak = sms * 4 * sm_mhz * 1e-3
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "G warp-instructions/s",
            "frac": achieved / peak, "warp_inst_per_launch": inst, "captured_tiles": source,
            "peak_kind": "SMs x 4 schedulers x 1 instruction per cycle at the sampled SM clock"}


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
    tune = None
    if args.no_autotune:
        if args.render_config:
            sim.set_render_config({**sim.render_config(), **json.loads(args.render_config)})
        best = sim.render_config()
    else:
        best, times = sim.autotune(ids, state, depth, rgb, iters=3)
        tune = {"{tile_w}x{tile_h}/rpl{rays_per_lane}/{s}stack{stack_depth}/{g}/bvh{node_width}".format(
                    s="smem" if c["stack_in_smem"] else "reg", g="staged" if c["stage_in_smem"] else "bcast", **c):
                round(t, 4) for c, t in zip(Sim.render_configs(), times)}
    for t in range(W):
        if t % EPISODE == 0:
            state.copy_(spawn)
        sim.step(state, cmds[t])
        sim.render(ids, state, depth, rgb)
    torch.cuda.synchronize()
    sim.check()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # no Python garbage collection inside the timed steps: a collection pause
    # between an event and the launches after it would show as GPU time
    gc.collect()
    gc.disable()
    with ClockSampler(dev.index if ws == 1 else local) as clk:
        for k in range(K):
            t = W + k
            if t % EPISODE == 0:
                state.copy_(spawn)
            flush.zero_()
            e0, e2 = ev[k]
            e0.record(stream)
            sim.step(state, cmds[t])
            sim.render(ids, state, depth, rgb)
            e2.record(stream)
        torch.cuda.synchronize()
    gc.enable()
    if ws > 1:
        dist.barrier()
    sim.check()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # Breakdown from a separate pass of the same loop with an event between the
    # dynamics and the render: that event itself costs about 3 us of the step,
    # which is why the timed loop above has none.
    evb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(min(K, 100))]
    state.copy_(spawn)
    for k, (e0, e1, e2) in enumerate(evb):
        t = W + k
        if t % EPISODE == 0:
            state.copy_(spawn)
        flush.zero_()
        e0.record(stream)
        sim.step(state, cmds[t])
        e1.record(stream)
        sim.render(ids, state, depth, rgb)
        e2.record(stream)
    torch.cuda.synchronize()
    dyn_ms = [a.elapsed_time(b) for a, b, c in evb]
    ren_ms = [b.elapsed_time(c) for a, b, c in evb]
    # The ray-cast kernel alone (the roofline's launch time): the library
    # records a CUDA event just before and just after the kernel, after its
    # estimate kernel, in every launch of one more pass of the same loop.
    state.copy_(spawn)
    sim.kernel_timing(True)
    for k in range(len(evb)):
        t = W + k
        if t % EPISODE == 0:
            state.copy_(spawn)
        flush.zero_()
        sim.step(state, cmds[t])
        sim.render(ids, state, depth, rgb)
    kern_ms = [float(x) for x in sim.kernel_times()]
    sim.kernel_timing(False)
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
    def e2e_loop(step):
        # Warm-up of at least 3 steps and 0.5 s: the host thread's per-step cost
        # (the enqueue of one step) settles only after a few hundred steps of
        # this loop, and a training loop runs at that settled rate.
        state.copy_(spawn)
        t_w, k = time.perf_counter(), 0
        while k < 3 or time.perf_counter() - t_w < E2E_WARMUP_S:
            if k % EPISODE == 0:
                state.copy_(spawn)
            step(k % (W + K))
            stream.synchronize()
            k += 1
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        gc.collect()
        gc.disable()
        t0 = time.perf_counter()
        for k in range(K2):
            if k % EPISODE == 0:
                state.copy_(spawn)
            step(W + k)
            stream.synchronize()        # the host reads the observation every step
        e2e_s = time.perf_counter() - t0
        gc.enable()
        if ws > 1:
            t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        return ws * n * K2 / e2e_s

    # the prepared step (one captured graph per call) is the value; the one-shot
    # sim_env_step call is reported beside it
    env = sim.make_env(ids, state, depth_h, rgb_h)
    prepared = e2e_loop(lambda t: env.step(cmd_host[t]))
    env.close()
    one_shot = e2e_loop(lambda t: sim.env_step(ids, state, cmd_host[t], depth_h, rgb_h))
    e2e = {"value": prepared, "unit": "agent-frames/s", "h2d_bytes_per_step": 4 * 4 * n,
           "d2h_bytes_per_step": n * p["height"] * p["width"] * 7, "steps": K2,
           "api": "Sim.make_env(...).step (sim_env_run) with page-locked host buffers",
           "warmup": f"at least 3 steps and {E2E_WARMUP_S} s of steps before the timed steps",
           "value_env_step": one_shot}

    # the batched and serving legs' scenes (and a 2M-triangle scene whose build
    # is timed) are generated on host cores while the GPU runs the extras below
    legs = ws == 1 and not args.no_extra_legs
    if legs:
        b_specs, s_specs = batched_specs(), serving_specs()
        pool = ScenePool(b_specs + s_specs + [BUILD_SCENE])

    # traversal counters of one launch -> algorithmic bytes of the ray-cast kernel
    state.copy_(spawn)
    sim.step(state, cmds[W])
    cnt = sim.render(ids, state, depth, rgb, counted=True)
    counted_states = state.T.double().cpu().numpy()   # the oracle's BVH walks the same rays (cpu_baseline leg)
    render_ms = statistics.mean(ren_ms)
    kernel_ms = statistics.mean(kern_ms)
    clocks = clk.summary()
    roof = raycast_roofline(sim, cnt, n, p, kernel_ms, clocks.get("sm_mhz"), best)
    roof["render_ms"] = render_ms
    roof["frac_of_render"] = roof["achieved"] * kernel_ms / render_ms / roof["peak"]

    # nearest-obstacle query (the paper's obstacle-distance module) on the same
    # agents: 20 calls captured in a CUDA graph, so the device time is measured
    # without the host's per-call marshalling in between
    for _ in range(3):
        sim.nearest_obstacle(ids, state, 10.0)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for _ in range(20):
            sim.nearest_obstacle(ids, state, 10.0)
    graph.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    graph.replay()
    e1.record()
    torch.cuda.synchronize()
    near_ms = e0.elapsed_time(e1) / 20
    del graph

    # the other rows on the path: the sensor epilogue and the other controllers
    state.copy_(spawn)
    sim.step(state, cmds[W])
    sensors = sensor_extra(sim, scene, sid, ids, state, depth, rgb, flush, n, p)
    controllers = controller_extra(sim, p, spawn, n, u_h)

    line = {"metric": METRIC, "value": value, "unit": "agent-frames/s", "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": 1e3 * total_s / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (procedural scene, seeded spawns and commands)",
            "config": {"workload": "single large scene: 208,812 triangles, 256 agents per GPU, RK4 dt=0.02, "
                                   "64x64 FP32 depth + uint8 RGB", "agents_per_gpu": n,
                       "triangles": int(scene.n_tris), "l2": "flushed between timed steps (256 MiB write)",
                       "reset_every_steps": EPISODE, "render_config": best, "autotune_ms": tune,
                       "bvh_depth": sim.scene_info(sid)["depth"]},
            "e2e": e2e, "gpu_launches": 3 * K,   # per step: dynamics, tile-cost estimate, ray cast
            "breakdown_ms": {"dynamics": statistics.mean(dyn_ms), "render": render_ms, "raycast_kernel": kernel_ms,
                             "from": "a separate pass of %d steps with an event between the two; the ray-cast "
                                     "kernel alone from a third pass with events around it "
                                     "(sim_kernel_timing)" % len(evb)},
            "roofline": roof,
            "extras": {"nearest_obstacle": {"agents": n, "ms": near_ms, "queries_per_s": n / (near_ms * 1e-3)},
                       "sensors": sensors, "controllers": controllers},
            "clocks": clocks}
    line["extras"]["build_ms"] = {"triangles_%d" % scene.n_tris: sim.scene_build_times(sid)}
    sim.close()
    if legs:
        # the bounded batched and serving legs of the same metric (sub-records)
        scenes_all = pool.result()
        pool.close()
        nb, ns = len(b_specs), len(s_specs)
        big = scenes_all[-1]
        with Sim(p) as bsim:
            bid = bsim.add_workload_scene(big)
            line["extras"]["build_ms"]["triangles_%d" % big.n_tris] = bsim.scene_build_times(bid)
        line["extras"]["build_ms"]["note"] = ("device time between stream events at the build's phase "
                                              "boundaries; wall = host time of sim_create_scene")
        bl = batched_leg(p, scenes_all[:nb], BATCHED_LOOPS, 1, compare_fixed=False)
        bl["workload"] = BATCHED_WORKLOAD
        bl["note"] = "%d timed graph launches of 100 steps after 1 warm-up launch" % BATCHED_LOOPS
        line["batched"] = bl
        sv = serving_leg(p, scenes_all[nb:nb + ns], loads=(SERVE_LOAD,), duration=SERVE_SECONDS)
        lv = sv["levels"][str(SERVE_LOAD)]
        line["serving"] = {"workload": SERVING_WORKLOAD, "load": SERVE_LOAD, "seconds_of_arrivals": SERVE_SECONDS,
                           **lv, "capacity_agents": sv["capacity_agents"],
                           "triangles_total": sv["triangles_total"], "bvh_build_s": sv["bvh_build_s"]}
        line["p50_ms"], line["p99_ms"] = lv["p50_ms"], lv["p99_ms"]
        line["extras"]["scene_generation"] = {"scenes": len(scenes_all), "workers": pool.workers,
                                              "wall_s": pool.wall_s}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_leg(p, scene, w_h, u_h, counted_states)
        line["roofline"]["per_ray"]["oracle_median_split"] = line["cpu_baseline"]["oracle_bvh_per_ray"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def multi_scene_cpu_baseline(p, scenes, w_h, u_h, n_pick=8, agents=2, steps=20, seed=77):
    """Oracle (as it stands) on a bounded sample of a multi-scene workload: two
    agents in each of eight seeded-random scenes, twenty steps of dynamics and
    render.  The oracle's own BVH builds are timed apart from the rate."""
    import oracle
    oracle.build()
    pick = sorted(np.random.default_rng(seed).choice(len(scenes), n_pick, replace=False).tolist())
    frames, t_used, build_s = 0, 0.0, 0.0
    for i in pick:
        t0 = time.perf_counter()
        osc = oracle.Scene.from_workload(scenes[i])
        build_s += time.perf_counter() - t0
        s = wl.spawn_states(scenes[i], agents, seed + i, w_h)
        cmds = wl.hover_commands(steps, agents, seed + 1000 + i, u_h)
        t0 = time.perf_counter()
        for t in range(steps):
            s = oracle.step(p, s, cmds[t])
            osc.render(p, s)
        t_used += time.perf_counter() - t0
        frames += agents * steps
    return {"value": frames / t_used, "unit": "agent-frames/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{agents} agents x {steps} steps in each of scenes {pick} (dynamics + render, FP64)",
            "oracle_bvh_build_s": build_s}


BATCHED_WORKLOAD = ("batched multi-scene: 64 scenes of 10k-1M triangles (log-uniform), 4,096 agents by Zipf(1.1), "
                    "100-step graph-captured loop, 64x64 depth+RGB")
SERVING_WORKLOAD = ("serving: 32 resident scenes of 50k-2M triangles, Poisson arrivals, 1-1024 agents x 1-16 steps "
                    "per request, last 64x64 depth+RGB returned")


def batched_specs(n_scenes=64, lo=10_000, hi=1_000_000, seed=99):
    """(triangles, seed) of the 64 procedural scenes with log-uniform triangle
    counts (seeds 100..163)."""
    sizes = wl.Rng(seed).log_uniform(lo, hi, n_scenes)
    return [(int(t), 100 + i) for i, t in enumerate(sizes)]


def serving_specs():
    """(triangles, seed) of the 32 resident scenes of 50k-2M triangles (seeds 500..531)."""
    sizes = wl.Rng(5).log_uniform(50_000, 2_000_000, 32)
    return [(int(t), 500 + i) for i, t in enumerate(sizes)]


class ScenePool:
    """Procedural scenes generated in spawned worker processes while the GPU
    works on something else.  The generator is plain numpy (no GPU, no CUDA
    state in the workers); spawn, not fork, because the parent holds a CUDA
    context."""

    def __init__(self, specs, workers=None):
        import concurrent.futures as cf
        import multiprocessing as mp
        workers = workers or max(1, min(len(specs), (os.cpu_count() or 2) - 2, 12))
        self.t0 = time.time()
        self.ex = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
        self.futs = [self.ex.submit(wl.sized_scene, t, sd) for t, sd in specs]
        self.workers = workers

    def result(self, lo=0, hi=None):
        out = [f.result() for f in self.futs[lo:hi]]
        self.wall_s = time.time() - self.t0
        return out

    def close(self):
        self.ex.shutdown(wait=True, cancel_futures=True)


BATCHED_AGENTS = 4096


def batched_groups(scenes, counts, w_h, pieces=None):
    """Spawn states of the batched workload: agent j of scene s is spawn state j
    of the seeded set of scene s, so a rank that runs agents first..first+count-1
    of a scene gets exactly the states the single-GPU run gives them.  pieces =
    [(scene, first, count)] (default: every agent of every scene); scenes maps a
    scene number to its mesh.  Returns [(scene, states [count, 17])]."""
    if pieces is None:
        pieces = [(s, 0, int(k)) for s, k in enumerate(counts)]
    return [(s, wl.spawn_states(scenes[s], int(counts[s]), 1000 + s, w_h)[a:a + c]) for s, a, c in pieces]


def batched_leg(p, scenes, steps, warmup, compare_fixed=True, iters_tune=3, groups=None, dist_ws=1, counts=None):
    """The batched multi-scene workload: 4,096 agents spread over the scenes by
    Zipf(1.1), one persistent render per step inside a graph-captured 100-step
    loop.  Returns the measurements (agent-frames/s of the autotuned
    configuration, and of the fixed 8x4 one when compare_fixed).  groups: this
    rank's [(scene, spawn states)] (default: all agents of all scenes); under
    torchrun (dist_ws > 1) every rank times its own groups and the value is the
    agents of all ranks over the slowest rank's time."""
    import torch
    from paper_2407_14783_b300.sim import Sim, to_soa
    w_h, u_h = _hover(p)
    T = 100
    if counts is None:
        counts = wl.zipf_partition(BATCHED_AGENTS, len(scenes), 1.1, 7)
    if groups is None:
        groups = batched_groups(scenes, counts, w_h)
    sim = Sim(p, device=torch.cuda.current_device())
    t0 = time.time()
    used = sorted({s for s, _ in groups})
    sid_of = {s: sim.add_workload_scene(scenes[s]) for s in used}
    sids = list(sid_of.values())
    torch.cuda.synchronize()
    build_s = time.time() - t0
    spawn = to_soa(np.concatenate([st for _, st in groups]))
    n_agents = spawn.shape[1]
    ids = torch.tensor(np.concatenate([np.full(len(st), sid_of[s]) for s, st in groups]), dtype=torch.int32,
                       device="cuda")
    cmds = torch.tensor(np.ascontiguousarray(wl.hover_commands(T, n_agents, 4, u_h).astype(np.float32)
                                             .transpose(0, 2, 1)), device="cuda")
    F = 2
    depth = torch.empty((F, n_agents, p["height"], p["width"]), device="cuda")
    rgb = torch.empty((F, n_agents, p["height"], p["width"], 3), dtype=torch.uint8, device="cuda")
    state = spawn.clone()
    fixed = sim.render_config()
    best, times = sim.autotune(ids, state, depth[0], rgb[0], iters=iters_tune)
    results = {}
    for name, cfg in ((("fixed_8x4", fixed),) if compare_fixed else ()) + (("autotuned", best),):
        sim.set_render_config(cfg)
        loop = sim.make_loop(ids, state, cmds, depth, rgb)
        for _ in range(warmup):
            state.copy_(spawn)
            loop.launch()
        torch.cuda.synchronize()
        if dist_ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
        evs = []
        with ClockSampler(torch.cuda.current_device()) as clk:
            for _ in range(steps):
                state.copy_(spawn)   # every timed loop starts from the spawn states (outside the events)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                loop.launch()
                e1.record()
                evs.append((e0, e1))
            torch.cuda.synchronize()
        sim.check()
        ms = [a.elapsed_time(b) for a, b in evs]
        frames, secs = n_agents * T * steps, sum(ms) * 1e-3
        if dist_ws > 1:
            from paper_2407_14783_b300.shard import reduce_step_metrics
            frames, secs = reduce_step_metrics(frames, secs)
        results[name] = {"clk": clk.summary(), "ms_per_loop": 1e3 * secs / steps, "value": frames / secs}
        loop.close()
    out = {"value": results["autotuned"]["value"], "unit": "agent-frames/s",
           "ms_per_step": results["autotuned"]["ms_per_loop"] / T, "loops": steps, "warmup_loops": warmup,
           "steps_per_loop": T, "agents": n_agents, "scenes": len(used),
           "triangles_total": int(sum(scenes[s].n_tris for s in used)),
           "triangles_min_max": [int(min(scenes[s].n_tris for s in used)), int(max(scenes[s].n_tris for s in used))],
           "agents_per_scene_min_max": [int(counts.min()), int(counts.max())],
           "scene_bytes": int(sum(sim.scene_info(i)["bytes"] for i in sids)),
           "bvh_depth_max": int(max(sim.scene_info(i)["depth"] for i in sids)),
           "autotuned_config": best, "bvh_build_s": build_s, "clocks": results["autotuned"]["clk"],
           "gpu_launches": steps * T * 3}   # per step: dynamics, tile-cost estimate, ray cast
    if compare_fixed:
        out["fixed_config"] = fixed
        out["fixed_value"] = results["fixed_8x4"]["value"]
        out["autotuned_over_fixed"] = results["autotuned"]["value"] / results["fixed_8x4"]["value"]
    sim.close()
    return out


def run_batched(args):
    """Batched multi-scene workload: 64 scenes of 10k-1M triangles, 4,096 agents
    spread by Zipf(1.1), one persistent render per step, 100-step graph-captured
    loop; autotuned render configuration against the fixed 8x4 one.  Under
    torchrun every rank builds and runs only its part of the plan_shards split
    (whole scenes, heavy scenes split by agents; no data-path collective)."""
    import torch
    ws, rank, local = _dist()
    p = wl.params()
    w_h, u_h = _hover(p)
    specs = batched_specs()
    counts = wl.zipf_partition(BATCHED_AGENTS, len(specs), 1.1, 7)
    if ws > 1:
        import torch.distributed as dist
        from paper_2407_14783_b300.shard import rank_workload
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        # an agent's render cost grows with the depth of its scene's BVH
        mine, pieces = rank_workload(counts, ws, rank, [math.log(t) for t, _ in specs])
    else:
        mine, pieces = list(range(len(specs))), None
    t0 = time.time()
    pool = ScenePool([specs[s] for s in mine])
    scenes = dict(zip(mine, pool.result()))
    pool.close()
    gen_s = time.time() - t0
    groups = batched_groups(scenes, counts, w_h, pieces)
    r = batched_leg(p, scenes, args.steps, args.warmup, compare_fixed=ws == 1, groups=groups, dist_ws=ws,
                    counts=counts)
    line = {"metric": METRIC, "value": r["value"], "unit": "agent-frames/s", "n_gpus": ws,
            "steps": args.steps * r["steps_per_loop"], "warmup": args.warmup * r["steps_per_loop"],
            "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "strong" if ws > 1 else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (64 procedural scenes, seeded)",
            "config": {"workload": BATCHED_WORKLOAD, "scenes": len(specs),
                       "triangles_total": int(sum(t for t, _ in specs)) if ws > 1 else r["triangles_total"],
                       "triangles_min_max": r["triangles_min_max"],
                       "agents_per_scene_min_max": r["agents_per_scene_min_max"],
                       "l2": "inputs larger than L2 (scene BVHs %.2f GB on rank 0)" % (r["scene_bytes"] / 1e9),
                       "autotuned_config": r["autotuned_config"],
                       "scene_generation_s": gen_s, "bvh_build_s": r["bvh_build_s"],
                       "bvh_depth_max": r["bvh_depth_max"],
                       "parallelism": "scene/agent shards (plan_shards), rank 0: %d scenes, %d agents" % (
                           r["scenes"], r["agents"]) if ws > 1 else "single GPU"},
            "gpu_launches": r["gpu_launches"], "clocks": r["clocks"]}
    if ws == 1:
        line["config"].update({"fixed_config": r["fixed_config"], "fixed_value": r["fixed_value"],
                               "autotuned_over_fixed": r["autotuned_over_fixed"]})
        if not getattr(args, "no_cpu_baseline", False):
            line["cpu_baseline"] = multi_scene_cpu_baseline(p, [scenes[s] for s in mine], w_h, u_h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def diff_cpu_baseline(p, s0, U, goals, lam, g0n, gcn, T, pick=(3, 517)):
    """Oracle (as it stands) on a bounded sample of the differentiable rollout:
    the exact FP64 gradient (forward-mode dual numbers) of two agents, timed,
    and the GPU gradient's error against it, as a whole vector and per
    component (relative, floored at 1e-3 of the agent's largest component)."""
    import oracle
    oracle.build()
    pick = np.asarray(pick)
    tg = time.perf_counter()
    Lr, gsr, gur = oracle.rollout_loss_grad(p, s0[pick].astype(np.float64), U[:, pick].astype(np.float64),
                                            goals[pick].astype(np.float64), lam)
    secs = time.perf_counter() - tg
    norm_err, comp_err = [], []
    for i, a in enumerate(pick):
        full = np.concatenate([g0n[a], gcn[:, a].ravel()])
        ref = np.concatenate([gsr[i], gur[:, i].ravel()])
        norm_err.append(float(np.linalg.norm(full - ref) / np.linalg.norm(ref)))
        scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
        comp_err.append(float((np.abs(full - ref) / scale).max()))
    return {"value": len(pick) * T / secs, "unit": "agent-steps/s (forward + exact gradient)",
            "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"agents {pick.tolist()} of the 1,024, all {T} steps, FP64 dual numbers",
            "gpu_grad_error": {"norm_relative": norm_err, "worst_component": comp_err}}


def run_diff(args):
    """Differentiable rollout: 1,024 agents, 200 steps at dt = 0.02, checkpoints
    every 10 steps; forward rollout kernel + hand-written adjoint kernel; loss =
    squared distance to seeded goals + 0.01 * control effort.  Reports agent-steps/s
    of forward + backward and the gradient error of sampled agents against the
    FP64 oracle's exact gradient."""
    import torch
    from paper_2407_14783_b300.sim import Sim, to_soa
    p = wl.params()
    w_h, u_h = _hover(p)
    scene = wl.cluttered_scene(seed=2)
    n, T, K, lam = 1024, 200, 10, 0.01
    s0 = wl.spawn_states(scene, n, 61, w_h).astype(np.float32)
    U = wl.hover_commands(T, n, 62, u_h, rate_range=0.3).astype(np.float32)
    goals = wl.goal_points(scene, n, 63).astype(np.float32)
    sim = Sim(p)
    st0 = to_soa(s0)
    cm = torch.tensor(np.ascontiguousarray(U.transpose(0, 2, 1)), device="cuda")
    g = torch.tensor(goals.T.copy(), device="cuda")
    fw, bw = [], []
    for it in range(args.warmup + args.steps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        states, ckpt, _ = sim.rollout(st0, cm, K=K)
        e1.record()
        gs = torch.zeros_like(states)
        gs[1:, 0:3] = 2.0 * (states[1:, 0:3] - g[None]) / T
        g0, gc = sim.rollout_backward(ckpt, cm, gs, K=K)
        gc += 2.0 * lam * cm / T
        e2.record()
        torch.cuda.synchronize()
        if it >= args.warmup:
            fw.append(e0.elapsed_time(e1))
            bw.append(e1.elapsed_time(e2))
    sim.check()
    g0n = g0.cpu().numpy().T
    gcn = gc.cpu().numpy().transpose(0, 2, 1)
    ms = statistics.mean(fw) + statistics.mean(bw)
    line = {"metric": "agent-steps/s (differentiable rollout: forward + adjoint) on 1 B300",
            "value": n * T / (ms * 1e-3), "unit": "agent-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / T, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded spawns, goals, commands)",
            "config": {"workload": "differentiable rollout: 1,024 agents, T=200, dt=0.02, checkpoint every 10 steps",
                       "forward_ms": statistics.mean(fw), "backward_ms": statistics.mean(bw),
                       "l2": "state 1024 x 17 floats, L2-resident"},
            "gpu_launches": 2}
    if not getattr(args, "no_cpu_baseline", False):
        line["cpu_baseline"] = diff_cpu_baseline(p, s0, U, goals, lam, g0n, gcn, T)
    print(json.dumps(line), flush=True)
    sim.close()
    return 0


def swarm_case(p, scene, n_form, steps, warmup, per=4, seed=71):
    """n_form formations of `per` drones (1.5 m square, common heading) flying
    through the scene as one swarm.  Returns (ms per step with the drones
    visible + proximity, ms per step in the parallel-agents mode, drone pixel
    fraction)."""
    import torch
    from paper_2407_14783_b300.sim import Sim, to_soa
    w_h, u_h = _hover(p)
    n = n_form * per
    lead = wl.spawn_states(scene, n_form, seed, w_h)
    s0 = np.repeat(lead, per, axis=0)
    offs = np.array([[0.75, 0.75], [0.75, -0.75], [-0.75, 0.75], [-0.75, -0.75]])
    for f in range(n_form):
        yaw = 2.0 * np.arctan2(lead[f, 9], lead[f, 6])
        c, sn = np.cos(yaw), np.sin(yaw)
        for k in range(per):
            s0[f * per + k, 0] += c * offs[k, 0] - sn * offs[k, 1]
            s0[f * per + k, 1] += sn * offs[k, 0] + c * offs[k, 1]
    s0 = s0.astype(np.float32)
    T = warmup + steps
    U = wl.hover_commands(T, n, seed + 1, u_h, rate_range=0.3).astype(np.float32)
    sim = Sim(p)
    sid = sim.add_workload_scene(scene)
    ids = torch.full((n,), sid, dtype=torch.int32, device="cuda")
    spawn = to_soa(s0)
    cmds = torch.tensor(np.ascontiguousarray(U.transpose(0, 2, 1)), device="cuda")
    d, c, h = sim.alloc_images(n, hit=True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    half, radius = (0.25, 0.25, 0.06), 0.3
    stream = torch.cuda.current_stream()

    def loop(swarm):
        sim.set_swarm(half if swarm else None, (250, 20, 30), 1000)
        state = spawn.clone()
        times = []
        for t in range(T):
            if t % 25 == 0:
                state.copy_(spawn)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(state, cmds[t])
            sim.render(ids, state, d, c, h)
            if swarm:
                sim.swarm_proximity(ids, state, radius)
            e1.record(stream)
            if t >= warmup:
                times.append((e0, e1))
        torch.cuda.synchronize()
        sim.check()
        return statistics.mean(a.elapsed_time(b) for a, b in times)

    ms_swarm = loop(True)
    drone_px = float((h < -1).float().mean().item())
    ms_plain = loop(False)
    sim.close()
    return ms_swarm, ms_plain, drone_px


def run_swarm(args):
    """Multi-agent mode (Sec. III-B): 256 agents flying in 64 formations of 4
    (1.5 m square, common heading) through the 208,812-triangle scene, all one
    swarm, so each camera also sees the other drones.  One step = dynamics +
    swarm render + pairwise proximity (collision query).  Reports agent-frames/s
    and the same loop in the parallel-agents mode beside it, and the same for
    swarms of 1,024 and 4,096 drones in the scene (the per-tile cull passes over
    every member of the swarm, so its cost grows with the swarm)."""
    p = wl.params()
    scene = wl.cluttered_scene(seed=2)
    half, radius = (0.25, 0.25, 0.06), 0.3
    ms_swarm, ms_plain, drone_px = swarm_case(p, scene, 64, args.steps, args.warmup)
    sweep = {}
    for n_form in (256, 1024):
        a, b, px = swarm_case(p, scene, n_form, args.steps, args.warmup)
        sweep[str(4 * n_form)] = {"swarm_ms_per_step": a, "parallel_ms_per_step": b, "swarm_over_parallel_time": a / b,
                                  "agent_frames_per_s": 4 * n_form / (a * 1e-3), "drone_pixel_fraction": px}
    n = 256
    line = {"metric": "agent-frames/s (dynamics+64x64 depth/RGB, multi-agent mode) on 1 B300",
            "value": n / (ms_swarm * 1e-3), "unit": "agent-frames/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_swarm, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (procedural scene, seeded formations)",
            "config": {"workload": "swarm: 256 agents in 64 formations of 4 as one swarm in the 208,812-triangle "
                                   "scene; step = dynamics + render with the other drones visible + proximity",
                       "drone_half_extents_m": half, "collision_radius_m": radius,
                       "drone_pixel_fraction": drone_px, "parallel_mode_ms_per_step": ms_plain,
                       "swarm_over_parallel_time": ms_swarm / ms_plain,
                       "l2": "flushed between timed steps (256 MiB write)"},
            "swarm_sizes": sweep,
            "gpu_launches": 6 * args.steps}   # per step: dynamics, swarm prep, estimate, ray cast, 2 proximity
    print(json.dumps(line), flush=True)
    return 0


class _PinnedArena:
    """Ring allocator over one pinned host buffer: request inputs and outputs
    for the load generator (allocation blocks while the oldest live block is in
    the way)."""

    def __init__(self, nbytes):
        import torch
        self.buf = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
        self.size = nbytes
        self.head = 0
        self.live = []          # (start, end, ticket) in allocation order

    def alloc(self, nbytes, release):
        nbytes = (nbytes + 255) & ~255
        if nbytes > self.size:
            raise MemoryError("arena too small")
        if self.head + nbytes > self.size:
            self.head = 0
        while self.live and self._overlaps(self.head, self.head + nbytes):
            release(self.live.pop(0)[2])
        start = self.head
        self.head += nbytes
        return start, start + nbytes

    def _overlaps(self, a, b):
        s, e, _ = self.live[0]
        return a < e and s < b

    def view(self, start, shape, dtype):
        import torch
        n = int(np.prod(shape)) * torch.tensor([], dtype=dtype).element_size()
        return self.buf[start:start + n].view(dtype).view(*shape)


def serving_leg(p, scenes, loads=(0.25, 0.5, 1.0), duration=3.0, rate=2000.0, cap=8192):
    """The serving workload: the scenes stay resident; Poisson arrivals (mean
    `rate` requests/s at load 1.0), each request n ~ log-U[1, 1024] agents of one
    scene for U{1..16} steps, returning the final state and the last 64x64 depth
    + RGB.  Throughput and p50 / p99 request latency per load level."""
    import torch
    from paper_2407_14783_b300.serve import Server
    from paper_2407_14783_b300.sim import Sim
    w_h, u_h = _hover(p)
    sim = Sim(p)
    t0 = time.time()
    sids = [sim.add_workload_scene(sc) for sc in scenes]
    build_s = time.time() - t0
    srv = Server(sim, capacity=cap)
    # per-scene pools of spawn states and commands (requests use the first n agents)
    pool_s = [np.ascontiguousarray(wl.spawn_states(sc, 1024, 600 + i, w_h).astype(np.float32).T)
              for i, sc in enumerate(scenes)]
    pool_u = np.ascontiguousarray(wl.hover_commands(16, 1024, 7, u_h).astype(np.float32).transpose(0, 2, 1))
    arena = _PinnedArena(6 << 30)
    H, W = p["height"], p["width"]
    levels = {}
    lat = {}

    def release(ticket):
        if ticket not in lat:
            lat[ticket] = srv.wait(ticket, 600000)

    for load in loads:
        li = {0.25: 0, 0.5: 1, 1.0: 2}.get(load, 3)
        reqs = wl.poisson_requests(rate * load, duration, len(scenes), 50 + li)
        arena.live.clear()
        arena.head = 0
        st0 = srv.stats()
        tickets = []
        start = time.perf_counter()
        for q in reqs:
            n, T = q["agents"], q["steps"]
            nb = 4 * (17 * n + T * 4 * n + 17 * n + n * H * W) + 3 * n * H * W
            delay = start + q["t"] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            a0, a1 = arena.alloc(nb, release)     # may wait for the oldest request in the way
            off = a0
            s0 = arena.view(off, (17, n), torch.float32); off += 4 * 17 * n
            cm = arena.view(off, (T, 4, n), torch.float32); off += 4 * T * 4 * n
            so = arena.view(off, (17, n), torch.float32); off += 4 * 17 * n
            do = arena.view(off, (n, H, W), torch.float32); off += 4 * n * H * W
            ro = arena.view(off, (n, H, W, 3), torch.uint8)
            s0.copy_(torch.from_numpy(pool_s[q["scene"]][:, :n]))
            cm.copy_(torch.from_numpy(pool_u[:T, :, :n]))
            tk = srv.submit(sids[q["scene"]], s0, cm, so, do, ro, frames="last")
            tickets.append(tk)
            arena.live.append((a0, a1, tk))
        for tk in tickets:
            release(tk)
        wall = time.perf_counter() - start
        st1 = srv.stats()
        lats = np.array([lat[t] for t in tickets])
        frames = sum(q["agents"] * q["steps"] for q in reqs)
        levels[str(load)] = {"offered_req_per_s": rate * load, "requests": len(reqs),
                             "offered_agent_frames_per_s": frames / duration,
                             "throughput_agent_frames_per_s": frames / wall,
                             "p50_ms": float(np.percentile(lats, 50)), "p99_ms": float(np.percentile(lats, 99)),
                             "mean_batch_agents": (st1["agent_frames"] - st0["agent_frames"]) /
                                                  max(1, st1["iterations"] - st0["iterations"]),
                             "wall_s": wall}
    srv.close()
    sim.close()
    return {"levels": levels, "triangles_total": int(sum(sc.n_tris for sc in scenes)), "capacity_agents": cap,
            "seconds_per_load": duration, "bvh_build_s": build_s}


def run_serving(args):
    """Serving workload: 32 resident scenes of 50k-2M triangles; Poisson arrivals
    (mean 2,000 requests/s at load 1.0), each request n ~ log-U[1, 1024] agents of one
    scene for U{1..16} steps, returning the final state and the last 64x64
    depth + RGB; throughput and p50 / p99 latency at loads 0.25, 0.5 and 1.0."""
    p = wl.params()
    w_h, u_h = _hover(p)
    t0 = time.time()
    pool = ScenePool(serving_specs())
    scenes = pool.result()
    pool.close()
    gen_s = time.time() - t0
    r = serving_leg(p, scenes, duration=float(args.serve_seconds))
    levels = r["levels"]
    full = levels["1.0"]
    line = {"metric": "agent-frames/s served (dynamics+64x64 depth/RGB) on 1 B300; p50/p99 step latency",
            "value": full["throughput_agent_frames_per_s"], "unit": "agent-frames/s", "n_gpus": 1,
            "steps": sum(v["requests"] for v in levels.values()), "warmup": 0,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (32 procedural scenes, Poisson request stream, seeded)",
            "config": {"workload": SERVING_WORKLOAD, "triangles_total": r["triangles_total"],
                       "capacity_agents": r["capacity_agents"], "seconds_per_load": r["seconds_per_load"],
                       "scene_generation_s": gen_s, "bvh_build_s": r["bvh_build_s"]},
            "served": levels, "p50_ms": full["p50_ms"], "p99_ms": full["p99_ms"]}
    if not getattr(args, "no_cpu_baseline", False):
        line["cpu_baseline"] = multi_scene_cpu_baseline(p, scenes, w_h, u_h)
    print(json.dumps(line), flush=True)
    return 0


def run_build(args):
    """Scene builds alone: the 208,812-triangle room and a 2M-triangle scene,
    each built --steps times after --warmup builds; CUDA-event time per build
    phase (mean over the timed builds) and the host time of the whole call."""
    import torch
    from paper_2407_14783_b300.sim import Sim
    p = wl.params()
    out = {}
    for name, scene in (("triangles_208812", make_workload(0)[1]), ("triangles_2M", wl.sized_scene(*BUILD_SCENE))):
        with Sim(p) as sim:
            runs = []
            for k in range(args.warmup + args.steps):
                sid = sim.add_workload_scene(scene)
                torch.cuda.synchronize()
                if k >= args.warmup:
                    runs.append(sim.scene_build_times(sid))
                sim.remove_scene(sid)
            out[name] = {ph: statistics.mean(r[ph] for r in runs) for ph in runs[0]}
            out[name]["n_tris"] = int(scene.n_tris)
    line = {"metric": "scene build time (ms)", "value": out["triangles_208812"]["wall"], "unit": "ms",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "dtype": "f32", "data": "synthetic (procedural scenes, seeded)",
            "config": {"workload": "BVH builds of the 208,812-triangle room and a 2M-triangle scene"},
            "build_ms": out}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing leg")
    ap.add_argument("--no-autotune", action="store_true", help="use the default ray-cast configuration")
    ap.add_argument("--render-config", default=None,
                    help="with --no-autotune: JSON fields that replace the default ray-cast configuration's, "
                         "e.g. '{\"stack_depth\": 32}'")
    ap.add_argument("--no-extra-legs", action="store_true",
                    help="skip the bounded batched and serving legs and the 2M-triangle build of the default run")
    ap.add_argument("--serve-seconds", type=float, default=3.0, help="seconds of arrivals per load level")
    ap.add_argument("--workload", choices=["large", "batched", "diff", "serving", "swarm", "build"], default="large",
                    help="large: single 208,812-triangle scene, 256 agents (default); batched: 64 scenes, "
                         "4,096 agents, graph-captured 100-step loop (--steps counts loops)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "diff":
        return run_diff(args)
    if args.workload == "swarm":
        return run_swarm(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "build":
        return run_build(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
