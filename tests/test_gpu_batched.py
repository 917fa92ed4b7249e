"""Batching pattern: many scenes of uneven size in one launch, and the
graph-captured step loop (Sec. III-D: several scenes run together)."""
import numpy as np
import pytest
import torch

from parity import compare_images

pytestmark = pytest.mark.gpu


def _setup(make_sim, wl, sizes, n_agents, seed=0):
    from paper_2407_14783_b300.sim import to_soa
    p = wl.params()
    sim = make_sim(p)
    scenes = [wl.sized_scene(t, 200 + seed + i) for i, t in enumerate(sizes)]
    sids = [sim.add_workload_scene(s) for s in scenes]
    counts = wl.zipf_partition(n_agents, len(scenes), 1.1, 7 + seed)
    states = [wl.spawn_states(s, int(k), 300 + seed + i, 1100.0).astype(np.float32)
              for i, (s, k) in enumerate(zip(scenes, counts))]
    all_s = np.concatenate(states)
    ids = torch.tensor(np.repeat(sids, counts), dtype=torch.int32, device="cuda")
    return p, sim, scenes, sids, counts, all_s, ids


def test_batched_multi_scene_sampled_parity(make_sim, oracle_mod, wl):
    """8 scenes of 2k-120k triangles, 512 agents spread by Zipf(1.1), one launch;
    two sampled agents per scene checked against the oracle."""
    from paper_2407_14783_b300.sim import to_soa
    sizes = [2000, 5000, 9000, 20000, 35000, 60000, 90000, 120000]
    p, sim, scenes, sids, counts, all_s, ids = _setup(make_sim, wl, sizes, 512)
    d, c, h = sim.alloc_images(all_s.shape[0], hit=True)
    sim.render(ids, to_soa(all_s), d, c, h)
    torch.cuda.synchronize()
    sim.check()
    d, c, h = d.cpu().numpy(), c.cpu().numpy(), h.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(counts)])
    rng = np.random.default_rng(5)
    for k, sc in enumerate(scenes):
        pick = off[k] + rng.choice(int(counts[k]), min(2, int(counts[k])), replace=False)
        compare_images(oracle_mod.Scene.from_workload(sc), p, all_s[pick].astype(np.float64), d[pick], c[pick],
                       h[pick])


def test_graph_loop_equals_eager_loop(make_sim, wl):
    """The captured T-step loop gives bit-identical states and frames to T eager
    (step, render) calls, and a second replay continues from the new state."""
    from paper_2407_14783_b300.sim import to_soa
    p, sim, scenes, sids, counts, all_s, ids = _setup(make_sim, wl, [3000, 8000, 15000], 90, seed=1)
    n = all_s.shape[0]
    T, F = 7, 3
    cmds = torch.stack([to_soa(u) for u in wl.hover_commands(T, n, 9, -0.6).astype(np.float32)])
    s0 = to_soa(all_s)
    # eager
    st = s0.clone()
    de = torch.zeros((F, n, 64, 64), device="cuda")
    ce = torch.zeros((F, n, 64, 64, 3), dtype=torch.uint8, device="cuda")
    for rep in range(2):
        for t in range(T):
            sim.step(st, cmds[t])
            sim.render(ids, st, de[t % F], ce[t % F])
        if rep == 0:
            st_eager1, de1, ce1 = st.clone(), de.clone(), ce.clone()
    torch.cuda.synchronize()
    # captured
    sl = s0.clone()
    dl = torch.zeros_like(de)
    cl = torch.zeros_like(ce)
    loop = sim.make_loop(ids, sl, cmds, dl, cl)
    loop.launch()
    torch.cuda.synchronize()
    assert torch.equal(sl, st_eager1) and torch.equal(dl, de1) and torch.equal(cl, ce1)
    loop.launch()
    torch.cuda.synchronize()
    assert torch.equal(sl, st) and torch.equal(dl, de) and torch.equal(cl, ce)
    loop.close()
    sim.check()


def test_autotune_picks_a_listed_config_and_images_match(make_sim, wl):
    from paper_2407_14783_b300.sim import Sim, to_soa
    p, sim, scenes, sids, counts, all_s, ids = _setup(make_sim, wl, [4000, 30000], 64, seed=2)
    st = to_soa(all_s)
    d0, c0, _ = sim.alloc_images(all_s.shape[0])
    sim.render(ids, st, d0, c0)
    d1, c1, _ = sim.alloc_images(all_s.shape[0])
    best, times = sim.autotune(ids, st, d1, c1, iters=2)
    assert best in Sim.render_configs()
    assert all(t > 0 for t in times)
    sim.render(ids, st, d1, c1)
    torch.cuda.synchronize()
    assert torch.equal(d0, d1) and torch.equal(c0, c1)
