"""Segmentation image and fused sensor noise against the oracle."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

NOISE = {"seed": 1234, "first_frame": 5, "depth_gauss": 0.02, "depth_speckle": 0.01, "depth_shot": 50.0,
         "depth_salt_pepper": 0.01, "rgb_gauss": 3.0, "rgb_speckle": 0.02, "rgb_shot": 0.5, "rgb_salt_pepper": 0.01,
         "seg_dropout": 0.05, "seg_gauss": 0.8, "seg_speckle": 0.01, "seg_shot": 2.0, "seg_salt_pepper": 0.02,
         "seg_max": 60}


def _unrounded_labels(onoise, cfg, n, seg_clean):
    """The oracle's segmentation labels after noise, before rounding (only the
    boundary test needs them; misses and dropped pixels are far from .5)."""
    H, W = seg_clean.shape[1:]
    b = onoise.counter_base(cfg["first_frame"], n, np.arange(n), H, W)
    return onoise._noisy(seg_clean.astype(np.float64), float(cfg["seg_max"]), cfg["seg_gauss"], cfg["seg_speckle"],
                         cfg["seg_shot"], cfg["seg_salt_pepper"], cfg["seed"], b + np.uint64(onoise.SEG_BLOCK))


def _setup(make_sim, wl):
    from paper_2407_14783_b300.sim import to_soa
    p = wl.params()
    sc = wl.room_scene()
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    labels = np.arange(sc.n_tris, dtype=np.int32) // 12          # room = 0, box k = k + 1
    sim.set_labels(sid, labels)
    n = 6
    s = wl.spawn_states(sc, n, 31, 1100.0).astype(np.float32)
    ids = torch.full((n,), sid, dtype=torch.int32, device="cuda")
    return p, sc, sim, labels, s, to_soa(s), ids


def _render(sim, ids, st, n):
    d, c, h = sim.alloc_images(n, hit=True)
    g = torch.empty_like(h)
    sim.render_seg(ids, st, d, c, h, g)
    torch.cuda.synchronize()
    sim.check()
    return d.cpu().numpy(), c.cpu().numpy(), h.cpu().numpy(), g.cpu().numpy()


def test_segmentation_labels(make_sim, oracle_mod, wl):
    p, sc, sim, labels, s, st, ids = _setup(make_sim, wl)
    d, c, h, g = _render(sim, ids, st, s.shape[0])
    r = oracle_mod.Scene.from_workload(sc).render(p, s.astype(np.float64))
    clear = ~r["tie"]
    ref = np.where(r["id"] >= 0, labels[np.maximum(r["id"], 0)], -1)
    assert np.array_equal(g[clear], ref[clear])
    assert np.array_equal(g, np.where(h >= 0, labels[np.maximum(h, 0)], -1))


def test_noise_matches_oracle_and_is_reproducible(make_sim, oracle_mod, wl):
    from oracle import noise as onoise
    p, sc, sim, labels, s, st, ids = _setup(make_sim, wl)
    n = s.shape[0]
    d0, c0, h0, g0 = _render(sim, ids, st, n)          # clean
    sim.set_noise(NOISE)
    d1, c1, h1, g1 = _render(sim, ids, st, n)          # frame 5
    d2, c2, h2, g2 = _render(sim, ids, st, n)          # frame 6: new draws
    sim.set_noise(NOISE)
    d3, c3, h3, g3 = _render(sim, ids, st, n)          # frame 5 again
    assert np.array_equal(d1, d3) and np.array_equal(c1, c3) and np.array_equal(g1, g3)
    assert not np.array_equal(d1, d2)
    assert np.array_equal(h1, h2)                      # hit ids are never noisy
    r = oracle_mod.Scene.from_workload(sc).render(p, s.astype(np.float64))
    seg_clean = np.where(r["id"] >= 0, labels[np.maximum(r["id"], 0)], -1)
    dn, cn, sn = onoise.apply(NOISE, 5, n, np.arange(n), r["depth"], r["rgb"], seg_clean, p["max_depth"])
    clear = ~r["tie"]
    assert np.all(np.abs(d1[clear] - dn[clear]) <= 1e-4 * (1.0 + dn[clear]))
    # colour is rounded from a float: at most one unit away, and only where the
    # unrounded oracle value sits near a rounding boundary
    diff = np.abs(c1.astype(int) - np.rint(cn).astype(int))
    assert diff[clear].max() <= 1
    near = np.abs(cn - np.floor(cn) - 0.5) < 1e-3
    assert not np.any((diff == 1) & clear[..., None] & ~near)
    # labels are rounded from a float as well: exact away from rounding
    # boundaries of the unrounded oracle label, else at most one apart
    su = _unrounded_labels(onoise, NOISE, n, seg_clean)
    snear = np.abs(su - np.floor(su) - 0.5) < 1e-3
    sdiff = np.abs(g1.astype(np.int64) - sn.astype(np.int64))
    assert np.all(sdiff[clear & ~snear] == 0) and sdiff[clear].max() <= 1
    sim.set_noise(None)
    out = _render(sim, ids, st, n)
    for a, b in zip(out, (d0, c0, h0, g0)):
        assert np.array_equal(a, b)
