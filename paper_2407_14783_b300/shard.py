"""Sharding of the rollout step across GPUs (one process per GPU).

Agents never interact in the parallel-agents mode (Sec. III-B), so the step
needs no per-step exchange: each rank steps and renders its own agents in its
own copies of the scenes those agents use.  This module plans the split and
provides the few collectives that sit outside the step: reducing benchmark
counters, gathering observations for a learner on one rank, and summing
gradients of the differentiable rollout.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Shard:
    """Agents of one rank: for each scene id, (first, count) ranges of that
    scene's agents (agent numbering within the scene)."""
    rank: int
    ranges: dict = field(default_factory=dict)
    cost: float = 0.0

    @property
    def scenes(self):
        return sorted(self.ranges)

    @property
    def n_agents(self) -> int:
        return int(sum(c for rs in self.ranges.values() for _, c in rs))


def plan_shards(agents_per_scene, world: int, scene_cost=None) -> list:
    """Split agents across `world` ranks.

    Work of an agent in scene s is scene_cost[s] (default 1).  Whole scenes go to
    the least-loaded rank, heaviest first; a scene whose work exceeds the even
    share is split by agents into pieces no larger than the share, so that every
    rank holds few scenes and the load stays within one piece of even.
    """
    counts = np.asarray(agents_per_scene, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    cost = np.ones(len(counts)) if scene_cost is None else np.asarray(scene_cost, dtype=float)
    work = counts * cost
    share = work.sum() / world if work.sum() > 0 else 0.0
    pieces = []  # (work, scene, first, count)
    for s in np.argsort(-work, kind="stable"):
        n = int(counts[s])
        if n == 0:
            continue
        per_agent = cost[s]
        if share > 0 and work[s] > share:
            k = int(np.ceil(work[s] / share))
            bounds = np.linspace(0, n, k + 1).round().astype(int)
            for a, b in zip(bounds[:-1], bounds[1:]):
                if b > a:
                    pieces.append(((b - a) * per_agent, int(s), int(a), int(b - a)))
        else:
            pieces.append((n * per_agent, int(s), 0, n))
    pieces.sort(key=lambda x: (-x[0], x[1], x[2]))
    shards = [Shard(r) for r in range(world)]
    for w, s, a, c in pieces:
        tgt = min(shards, key=lambda sh: (sh.cost, sh.rank))
        tgt.ranges.setdefault(s, []).append((a, c))
        tgt.cost += w
    return shards


def local_agents(shard: Shard, agents_per_scene) -> list:
    """(scene, agent index within the scene) pairs of a shard, in scene order."""
    out = []
    for s in shard.scenes:
        for a, c in shard.ranges[s]:
            out.extend((s, a + j) for j in range(c))
    return out


def rank_workload(agents_per_scene, world: int, rank: int, scene_cost=None):
    """The part of a multi-scene workload that one rank runs: the scenes it must
    build (sorted) and its agent pieces as (scene, first, count), from the same
    plan on every rank (plan_shards is deterministic), so no exchange is needed
    to agree on it."""
    shard = plan_shards(agents_per_scene, world, scene_cost)[rank]
    pieces = [(s, a, c) for s in shard.scenes for a, c in shard.ranges[s]]
    return shard.scenes, pieces


def reduce_step_metrics(frames: int, seconds: float, group=None):
    """Whole-job agent-frames and the slowest rank's time (max over ranks)."""
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else "cpu"
    f = torch.tensor([float(frames)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(f, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return int(f.item()), float(t.item())


def gather_to_rank0(local, group=None):
    """Concatenate every rank's local tensor (agents along dim 0) on rank 0, in rank
    order; other ranks get None.  For a learner that consumes observations."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n = torch.tensor([local.shape[0]], dtype=torch.int64, device=local.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    m = int(max(int(x.item()) for x in sizes))
    pad = torch.zeros((m,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    if dist.get_rank(group) != 0:
        return None
    return torch.cat([p[: int(s.item())] for p, s in zip(parts, sizes)], dim=0)


def allreduce_sum_(t, group=None):
    """In-place sum over ranks (e.g. gradients of a shared policy)."""
    import torch.distributed as dist
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t
