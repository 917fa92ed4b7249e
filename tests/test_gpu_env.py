"""The host-buffer environment step (sim_env_step): page-locked buffers that the
kernels read and write in place, and pageable buffers that go through device
staging, both give exactly the step + render of device buffers."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _case(make_sim, wl, n=37):
    from paper_2407_14783_b300.sim import to_soa
    p = wl.params()
    sc = wl.room_scene()
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    s0 = to_soa(wl.spawn_states(sc, n, 77, 1100.0).astype(np.float32))
    u_hover = 2 * p["g"] / p["a_max"] - 1
    cmds = torch.from_numpy(np.ascontiguousarray(wl.hover_commands(4, n, 78, u_hover).transpose(0, 2, 1)))
    cmds = cmds.float()                                    # [T][4][n]
    ids = torch.full((n,), sid, dtype=torch.int32, device="cuda")
    return p, sim, ids, s0, cmds


def _device_run(sim, ids, s0, cmds):
    st = s0.clone()
    n = st.shape[1]
    out = []
    for t in range(cmds.shape[0]):
        sim.step(st, cmds[t].cuda())
        d, c, _ = sim.alloc_images(n)
        sim.render(ids, st, d, c)
        out.append((d.cpu(), c.cpu(), st.cpu()))
    torch.cuda.synchronize()
    sim.check()
    return out


@pytest.mark.parametrize("pinned", [True, False])
def test_env_step_equals_device_step_and_render(make_sim, wl, pinned):
    p, sim, ids, s0, cmds = _case(make_sim, wl)
    n = s0.shape[1]
    ref = _device_run(sim, ids, s0, cmds)
    st = s0.clone()

    def host(t):
        return t.pin_memory() if pinned else t

    cmd_h = host(cmds.contiguous())
    depth_h = host(torch.full((n, p["height"], p["width"]), -7.0))
    rgb_h = host(torch.full((n, p["height"], p["width"], 3), 9, dtype=torch.uint8))
    state_h = host(torch.zeros((17, n)))
    stream = torch.cuda.current_stream()
    for t in range(cmds.shape[0]):
        sim.env_step(ids, st, cmd_h[t], depth_h, rgb_h, state_h)
        stream.synchronize()
        d, c, s = ref[t]
        assert torch.equal(depth_h, d) and torch.equal(rgb_h, c) and torch.equal(state_h, s)
    sim.check()


def test_env_step_without_images_only_steps(make_sim, wl):
    p, sim, ids, s0, cmds = _case(make_sim, wl, n=5)
    ref = _device_run(sim, ids, s0, cmds[:1])
    st = s0.clone()
    sim.env_step(ids, st, cmds[0].contiguous().pin_memory())
    torch.cuda.synchronize()
    sim.check()
    assert torch.equal(st.cpu(), ref[0][2])


@pytest.mark.parametrize("shape", [(8, 4, 1), (16, 2, 1), (8, 8, 2), (16, 4, 2)])
def test_streamed_download_tile_shapes_ragged_image_and_noise(make_sim, wl, shape):
    """Band completion counts pixels, so every tile shape, a last band shorter
    than a tile (38 rows) and the quarter-tile sub-packets all stream every
    pixel exactly once; noise is applied before the band leaves."""
    from paper_2407_14783_b300.sim import to_soa
    tw, th, rpl = shape
    p = wl.params(width=40, height=38)
    sc = wl.room_scene()
    sim = make_sim(p)
    cfg = sim.render_config()
    cfg.update(tile_w=tw, tile_h=th, rays_per_lane=rpl)
    sim.set_render_config(cfg)
    sid = sim.add_workload_scene(sc)
    n = 29
    s0 = to_soa(wl.spawn_states(sc, n, 91, 1100.0).astype(np.float32))
    ids = torch.full((n,), sid, dtype=torch.int32, device="cuda")
    cmd = torch.zeros((4, n))
    noise = {"seed": 3, "first_frame": 0, "depth_gauss": 0.01, "rgb_gauss": 2.0}
    sim.set_noise(noise)
    st = s0.clone()
    sim.step(st, cmd.cuda())
    d, c, _ = sim.alloc_images(n)
    for _ in range(3):                      # also exercises the scheduling hints of repeated launches
        sim.set_noise(noise)
        sim.render(ids, st, d, c)
    torch.cuda.synchronize()
    depth_h = torch.full((n, 38, 40), -1.0).pin_memory()
    rgb_h = torch.zeros((n, 38, 40, 3), dtype=torch.uint8).pin_memory()
    st2 = s0.clone()
    for _ in range(3):
        sim.set_noise(noise)
        sim.env_step(ids, st2, cmd.contiguous().pin_memory(), depth_h, rgb_h)
        st2.copy_(s0)
    torch.cuda.synchronize()
    sim.check()
    assert torch.equal(depth_h, d.cpu()) and torch.equal(rgb_h, c.cpu())


@pytest.mark.parametrize("pinned", [True, False])
def test_env_step_after_image_size_grows(make_sim, wl, pinned):
    """Staging and completion buffers follow the image size, not only the
    agent count: a larger image with the same agents after sim_set_params."""
    from paper_2407_14783_b300.sim import to_soa
    p = wl.params(width=32, height=32)
    sc = wl.room_scene()
    sim = make_sim(p)
    sid = sim.add_workload_scene(sc)
    n = 11
    s0 = to_soa(wl.spawn_states(sc, n, 5, 1100.0).astype(np.float32))
    ids = torch.full((n,), sid, dtype=torch.int32, device="cuda")
    cmd = torch.zeros((4, n))
    for size in (32, 96):
        p2 = wl.params(width=size, height=size)
        sim.set_params(p2)
        d_h = torch.zeros((n, size, size))
        c_h = torch.zeros((n, size, size, 3), dtype=torch.uint8)
        if pinned:
            d_h, c_h = d_h.pin_memory(), c_h.pin_memory()
        st = s0.clone()
        sim.env_step(ids, st, cmd.contiguous(), d_h, c_h)
        torch.cuda.synchronize()
        sim.check()
        d, c, _ = sim.alloc_images(n)
        st2 = s0.clone()
        sim.step(st2, cmd.cuda())
        sim.render(ids, st2, d, c)
        torch.cuda.synchronize()
        assert torch.equal(d_h, d.cpu()) and torch.equal(c_h, c.cpu())


@pytest.mark.parametrize("cmd_pinned", [True, False])
def test_prepared_env_equals_device_step_and_render(make_sim, wl, cmd_pinned):
    """sim_env_run (one captured graph per step, the command pointer rebound
    per call) gives exactly the step + render of device buffers, and the state
    download."""
    p, sim, ids, s0, cmds = _case(make_sim, wl)
    n = s0.shape[1]
    ref = _device_run(sim, ids, s0, cmds)
    st = s0.clone()
    depth_h = torch.full((n, p["height"], p["width"]), -7.0).pin_memory()
    rgb_h = torch.full((n, p["height"], p["width"], 3), 9, dtype=torch.uint8).pin_memory()
    state_h = torch.zeros((17, n)).pin_memory()
    env = sim.make_env(ids, st, depth_h, rgb_h, state_h)
    cmd_h = cmds.contiguous()
    if cmd_pinned:
        cmd_h = cmd_h.pin_memory()
    for t in range(cmds.shape[0]):
        env.step(cmd_h[t])
        torch.cuda.current_stream().synchronize()
        d, c, s = ref[t]
        assert torch.equal(depth_h, d) and torch.equal(rgb_h, c) and torch.equal(state_h, s)
    sim.check()
    env.close()


def test_prepared_env_picks_up_context_changes(make_sim, wl):
    """A change of noise, render configuration or multi-agent mode between runs
    is captured anew: the next run matches the device path under the new
    settings."""
    p, sim, ids, s0, cmds = _case(make_sim, wl, n=24)
    n = s0.shape[1]
    depth_h = torch.zeros((n, p["height"], p["width"])).pin_memory()
    rgb_h = torch.zeros((n, p["height"], p["width"], 3), dtype=torch.uint8).pin_memory()
    st = s0.clone()
    env = sim.make_env(ids, st, depth_h, rgb_h)
    noise = {"seed": 8, "first_frame": 3, "depth_gauss": 0.01, "rgb_gauss": 2.0}
    cfg = sim.render_config()
    changes = [lambda: sim.set_noise(noise), lambda: sim.set_noise(None),
               lambda: sim.set_render_config(dict(cfg, tile_w=16, tile_h=2)),
               lambda: sim.set_swarm((0.25, 0.18, 0.06), (250, 20, 30), 7)]
    for apply in changes:
        apply()
        ref = _device_run(sim, ids, s0, cmds[:1])
        apply()            # noise: back to its first frame, so both renders draw the same frame
        st.copy_(s0)
        env.step(cmds[0].contiguous().pin_memory())
        torch.cuda.synchronize()
        sim.check()
        assert torch.equal(depth_h, ref[0][0]) and torch.equal(rgb_h, ref[0][1])
    env.close()


def test_prepared_env_rejects_pageable_images(make_sim, wl):
    from paper_2407_14783_b300.binding import SimError
    p, sim, ids, s0, cmds = _case(make_sim, wl, n=4)
    with pytest.raises(SimError):
        sim.make_env(ids, s0.clone(), torch.zeros((4, p["height"], p["width"])))
