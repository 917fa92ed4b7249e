"""Multi-GPU layout on CPU: the shard plan and the collectives around the step,
exercised with world_size-2 gloo process groups (no GPU needed)."""
import os
import socket

import numpy as np


def test_plan_covers_every_agent_once_and_balances():
    from paper_2407_14783_b300.shard import plan_shards, local_agents
    rng = np.random.default_rng(0)
    for trial in range(50):
        ns = int(rng.integers(1, 40))
        counts = rng.integers(0, 300, ns)
        cost = rng.uniform(0.2, 5.0, ns)
        world = int(rng.integers(1, 9))
        shards = plan_shards(counts, world, cost)
        seen = {}
        for sh in shards:
            for s, a in local_agents(sh, counts):
                seen[(s, a)] = seen.get((s, a), 0) + 1
        assert sum(seen.values()) == counts.sum() and all(v == 1 for v in seen.values())
        assert set(seen) == {(s, a) for s in range(ns) for a in range(counts[s])}
        total = float((counts * cost).sum())
        if total > 0:
            share = total / world
            largest_piece = max(min(c * w, share) for c, w in zip(counts, cost) if c > 0)
            assert max(sh.cost for sh in shards) <= share + largest_piece + 1e-6


def test_plan_splits_one_heavy_scene():
    from paper_2407_14783_b300.shard import plan_shards
    shards = plan_shards([1000, 10, 10], 4)
    assert all(0 in sh.ranges for sh in shards)          # the heavy scene is on every rank
    assert max(sh.n_agents for sh in shards) - min(sh.n_agents for sh in shards) <= 20


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2407_14783_b300 import workloads as wl
    from paper_2407_14783_b300.shard import plan_shards, local_agents, gather_to_rank0, reduce_step_metrics, \
        allreduce_sum_
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = wl.params(width=16, height=12)
    scenes = [wl.room_scene(seed=1), wl.room_scene(seed=3)]
    counts = [5, 9]
    spawn = [wl.spawn_states(sc, c, 10 + i, 1100.0) for i, (sc, c) in enumerate(zip(scenes, counts))]
    cmds = [wl.uniform_commands(3, c, 20 + i) for i, c in enumerate(counts)]
    shard = plan_shards(counts, world)[rank]
    mine = local_agents(shard, counts)
    states, depths = [], []
    osc = {s: oracle.Scene.from_workload(scenes[s]) for s in shard.scenes}
    for s, a in mine:
        traj = oracle.rollout(p, spawn[s][a:a + 1], cmds[s][:, a:a + 1])
        states.append(traj[-1, 0])
        depths.append(osc[s].render(p, traj[-1])["depth"][0])
    key = torch.tensor([[s, a] for s, a in mine], dtype=torch.int64).reshape(-1, 2)
    st = torch.tensor(np.array(states)).reshape(-1, 17)
    dp = torch.tensor(np.array(depths)).reshape(-1, 12, 16)
    gk, gs, gd = gather_to_rank0(key), gather_to_rank0(st), gather_to_rank0(dp)
    frames, secs = reduce_step_metrics(len(mine) * 3, 0.5 + rank)
    g = torch.full((3,), float(rank + 1))
    allreduce_sum_(g)
    if rank == 0:
        torch.save({"key": gk, "state": gs, "depth": gd, "frames": frames, "secs": secs, "g": g}, out_path)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_step_and_gather_matches_single_process(tmp_path, oracle_mod, wl):
    import torch
    import torch.multiprocessing as mp
    out = str(tmp_path / "r0.pt")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    res = torch.load(out)
    p = wl.params(width=16, height=12)
    scenes = [wl.room_scene(seed=1), wl.room_scene(seed=3)]
    counts = [5, 9]
    assert res["frames"] == sum(counts) * 3 and res["secs"] == 1.5
    assert torch.equal(res["g"], torch.full((3,), 3.0))
    keys = [tuple(k) for k in res["key"].tolist()]
    assert sorted(keys) == [(s, a) for s in range(2) for a in range(counts[s])]
    for i, (s, a) in enumerate(keys):
        sp = wl.spawn_states(scenes[s], counts[s], 10 + s, 1100.0)
        cm = wl.uniform_commands(3, counts[s], 20 + s)
        ref = oracle_mod.rollout(p, sp[a:a + 1], cm[:, a:a + 1])[-1]
        assert np.array_equal(res["state"][i].numpy(), ref[0])
        dref = oracle_mod.Scene.from_workload(scenes[s]).render(p, ref)["depth"][0]
        assert np.array_equal(res["depth"][i].numpy(), dref)


def _batched_worker(rank, world, port, out_path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import math
    import torch
    import torch.distributed as dist
    from paper_2407_14783_b300 import workloads as wl
    from paper_2407_14783_b300.shard import rank_workload, plan_shards, reduce_step_metrics
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # the batched workload's split: 64 scenes of log-uniform 10k-1M triangles,
    # 4,096 agents by Zipf(1.1), cost per agent log(triangles)
    sizes = wl.Rng(99).log_uniform(10_000, 1_000_000, 64)
    counts = wl.zipf_partition(4096, 64, 1.1, 7)
    cost = [math.log(t) for t in sizes]
    scenes, pieces = rank_workload(counts, world, rank, cost)
    plan = plan_shards(counts, world, cost)[rank]
    assert scenes == plan.scenes
    assert sorted((s, a, c) for s in plan.ranges for a, c in plan.ranges[s]) == sorted(pieces)
    mine = torch.tensor(pieces, dtype=torch.int64).reshape(-1, 3)
    n = torch.tensor([mine.shape[0]])
    sizes_g = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes_g, n)
    m = int(max(int(x) for x in sizes_g))
    pad = torch.full((m, 3), -1, dtype=torch.int64)
    pad[: mine.shape[0]] = mine
    parts = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    frames, secs = reduce_step_metrics(int(sum(c for _, _, c in pieces)) * 100, 1.0 + rank)
    if rank == 0:
        torch.save({"parts": [p[: int(k)] for p, k in zip(parts, sizes_g)], "frames": frames, "secs": secs,
                    "counts": torch.tensor(counts)}, out_path)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_batched_split_covers_the_workload(tmp_path):
    """Each rank of a world-2 gloo group takes its part of the batched workload
    from the shared plan; together the parts hold every agent of every scene
    exactly once, and the reduced frame count is the whole workload's."""
    import torch
    import torch.multiprocessing as mp
    out = str(tmp_path / "split.pt")
    mp.start_processes(_batched_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    res = torch.load(out)
    counts = res["counts"].numpy()
    seen = {}
    for rank_part in res["parts"]:
        for s, a, c in rank_part.tolist():
            for j in range(a, a + c):
                seen[(s, j)] = seen.get((s, j), 0) + 1
    assert all(v == 1 for v in seen.values())
    assert set(seen) == {(s, j) for s in range(len(counts)) for j in range(int(counts[s]))}
    assert res["frames"] == int(counts.sum()) * 100 and res["secs"] == 2.0
    # both ranks hold work, and neither holds every scene
    assert all(0 < len({s for s, _, _ in p.tolist()}) < len(counts) for p in res["parts"])
