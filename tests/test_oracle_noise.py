"""Pins of the sensor-noise oracle: generator reference values and the
moments each noise model must have."""
import numpy as np


def test_generator_reference_values():
    from oracle.noise import splitmix64
    out = splitmix64(0, np.array([0, 1], np.uint64))
    assert int(out[0]) == 0xE220A8397B1DCDAF and int(out[1]) == 0x6E789E6AA1B965F4


def test_gaussian_moments():
    from oracle.noise import gauss
    z = gauss(7, np.arange(0, 400000, 2, dtype=np.uint64))
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01
    assert abs(np.mean(z ** 4) - 3.0) < 0.05           # normal kurtosis


def test_models_have_the_stated_moments():
    from oracle.noise import apply
    k, H, W = 4, 64, 64
    d = np.full((k, H, W), 5.0)
    rgb = np.full((k, H, W, 3), 100, np.uint8)
    seg = np.zeros((k, H, W), np.int32)
    agents = np.arange(k)
    g, _, _ = apply({"seed": 3, "depth_gauss": 0.1}, 0, k, agents, d, rgb, None, 10.0)
    assert abs(g.mean() - 5.0) < 0.005 and abs(g.std() - 0.1) < 0.005
    sp, _, _ = apply({"seed": 3, "depth_speckle": 0.05}, 0, k, agents, d, rgb, None, 10.0)
    assert abs(sp.std() - 0.25) < 0.01
    sh, _, _ = apply({"seed": 3, "depth_shot": 20.0}, 0, k, agents, d, rgb, None, 10.0)
    assert abs(sh.var() - 5.0 / 20.0) < 0.02            # var of (Poisson-like L) / k = x / k
    sa, _, _ = apply({"seed": 3, "depth_salt_pepper": 0.1}, 0, k, agents, d, rgb, None, 10.0)
    assert abs(np.mean(sa != 5.0) - 0.1) < 0.01
    assert abs(np.mean(sa == 0.0) - 0.05) < 0.01 and abs(np.mean(sa == 10.0) - 0.05) < 0.01
    _, c, s = apply({"seed": 3, "rgb_gauss": 4.0, "seg_dropout": 0.2}, 0, k, agents, d, rgb, seg, 10.0)
    assert abs(c.std() - 4.0) < 0.1 and abs(np.mean(s == -1) - 0.2) < 0.01
    # channels and frames draw from distinct counters
    assert np.corrcoef(c[..., 0].ravel(), c[..., 1].ravel())[0, 1] < 0.02
    g2, _, _ = apply({"seed": 3, "depth_gauss": 0.1}, 1, k, agents, d, rgb, None, 10.0)
    assert np.corrcoef(g.ravel(), g2.ravel())[0, 1] < 0.02


def test_slot_blocks_are_disjoint():
    """Every (image, model) pair draws from its own generator outputs: the blocks
    of depth, the three colour channels and segmentation, and the dropout slot,
    do not overlap and fit in the per-pixel stride."""
    from oracle import noise as nz
    used = []
    for base in (nz.DEPTH_BLOCK, nz.COLOUR_BLOCK, nz.COLOUR_BLOCK + 8, nz.COLOUR_BLOCK + 16, nz.SEG_BLOCK):
        used += range(base, base + 8)
    used.append(nz.SEG_DROPOUT)
    assert len(set(used)) == len(used) and max(used) < nz.STRIDE


def test_blue_salt_pepper_and_segmentation_dropout_are_independent():
    """P(both) = p^2 for independent draws; a shared draw would give p."""
    from oracle.noise import apply
    k, H, W = 8, 64, 64
    d = np.full((k, H, W), 5.0)
    rgb = np.full((k, H, W, 3), 100, np.uint8)
    seg = np.zeros((k, H, W), np.int32)
    _, c, s = apply({"seed": 9, "rgb_salt_pepper": 0.3, "seg_dropout": 0.3}, 0, k, np.arange(k), d, rgb, seg, 10.0)
    both = np.mean((c[..., 2] != 100) & (s == -1))
    assert abs(both - 0.09) < 0.01


def test_segmentation_label_noise():
    """Label noise keeps labels integral, inside [0, seg_max], and unlabelled
    pixels unlabelled; Gaussian label noise has the stated spread before
    rounding (variance sigma^2 + 1/12 after it)."""
    from oracle.noise import apply
    k, H, W = 8, 64, 64
    d = np.full((k, H, W), 5.0)
    rgb = np.zeros((k, H, W, 3), np.uint8)
    seg = np.full((k, H, W), 50, np.int32)
    seg[:, :, :4] = -1
    _, _, s = apply({"seed": 4, "seg_gauss": 3.0, "seg_max": 100}, 0, k, np.arange(k), d, rgb, seg, 10.0)
    lab = s[:, :, 4:]
    assert np.all(s[:, :, :4] == -1) and lab.min() >= 0 and lab.max() <= 100
    assert abs(lab.mean() - 50.0) < 0.1 and abs(lab.var() - (9.0 + 1.0 / 12.0)) < 0.3
    _, _, s2 = apply({"seed": 4, "seg_salt_pepper": 0.2, "seg_max": 100}, 0, k, np.arange(k), d, rgb, seg, 10.0)
    lab2 = s2[:, :, 4:]
    assert abs(np.mean(lab2 == 0) - 0.1) < 0.01 and abs(np.mean(lab2 == 100) - 0.1) < 0.01
