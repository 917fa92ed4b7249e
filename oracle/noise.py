"""Sensor-noise oracle (TEST INFRASTRUCTURE ONLY).

Applies the vision-sensor noise models of the paper's domain randomisation
(Sec. III-D, Table II: Gaussian, Poisson-type shot noise, salt and pepper,
speckle) to clean images, in float64 numpy, drawing every random number from
its own implementation of SplitMix64 (Steele, Lea and Flood 2014), indexed by
the counter layout stated with the library's noise configuration:
  i = ((frame * n_agents + agent) * H * W + pixel) * 64 + slot   (mod 2^64),
slots: depth 0-7, colour channel c 8 + 8c .. 15 + 8c, segmentation 32-39,
segmentation dropout 40; within a block of 8: Gaussian 0-1, speckle 2-3,
shot 4-5, salt and pepper 6-7.
Shares no code with the CUDA path.
"""
from __future__ import annotations

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)

STRIDE = 64                      # generator outputs reserved per pixel
DEPTH_BLOCK, COLOUR_BLOCK, SEG_BLOCK, SEG_DROPOUT = 0, 8, 32, 40


def splitmix64(seed: int, i: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(i, np.uint64) + np.uint64(1)) * _G
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _u_half_open(x):
    return (x >> np.uint64(40)).astype(np.float64) / 16777216.0


def _u_open(x):
    return ((x >> np.uint64(40)).astype(np.float64) + 0.5) / 16777216.0


def gauss(seed, i):
    """Standard normal from outputs i and i + 1 (Box-Muller, cosine branch)."""
    u1 = _u_open(splitmix64(seed, i))
    u2 = _u_half_open(splitmix64(seed, i + np.uint64(1)))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def _noisy(x, hi, g, sp, shot, sandp, seed, b):
    x = x.astype(np.float64).copy()
    if shot > 0:
        lam = shot * x
        x = (lam + np.sqrt(np.maximum(lam, 0.0)) * gauss(seed, b + np.uint64(4))) / shot
    if g > 0:
        x = x + g * gauss(seed, b)
    if sp > 0:
        x = x * (1.0 + sp * gauss(seed, b + np.uint64(2)))
    if sandp > 0:
        hit = _u_half_open(splitmix64(seed, b + np.uint64(6))) < np.float64(np.float32(sandp))
        val = np.where(_u_half_open(splitmix64(seed, b + np.uint64(7))) < 0.5, 0.0, hi)
        x = np.where(hit, val, x)
    return np.clip(x, 0.0, hi)


def counter_base(frame: int, n_agents: int, agents: np.ndarray, H: int, W: int) -> np.ndarray:
    """Base counters [len(agents), H, W] of the pixels of the given agents."""
    pix = np.arange(H * W, dtype=np.uint64).reshape(H, W)
    with np.errstate(over="ignore"):
        a = (np.uint64(frame) * np.uint64(n_agents) + np.asarray(agents, np.uint64))[:, None, None]
        return (a * np.uint64(H * W) + pix[None]) * np.uint64(STRIDE)


def apply(cfg: dict, frame: int, n_agents: int, agents, depth, rgb, seg, max_depth: float):
    """Noisy copies of clean images of the given agents (depth [k,H,W], rgb [k,H,W,3],
    seg [k,H,W] or None).  Returns (depth float64, rgb float64 before rounding, seg).

    Segmentation (Table II lists the same four models for it): a labelled pixel's
    label is perturbed as a number in [0, seg_max] and rounded half to even; an
    unlabelled pixel (-1) stays unlabelled; then dropout unlabels a pixel with
    probability seg_dropout."""
    seed = int(cfg.get("seed", 0))
    k, H, W = depth.shape
    b = counter_base(frame, n_agents, agents, H, W)
    d = _noisy(depth, max_depth, cfg.get("depth_gauss", 0), cfg.get("depth_speckle", 0), cfg.get("depth_shot", 0),
               cfg.get("depth_salt_pepper", 0), seed, b + np.uint64(DEPTH_BLOCK))
    c = np.stack([_noisy(rgb[..., ch].astype(np.float64), 255.0, cfg.get("rgb_gauss", 0), cfg.get("rgb_speckle", 0),
                         cfg.get("rgb_shot", 0), cfg.get("rgb_salt_pepper", 0), seed,
                         b + np.uint64(COLOUR_BLOCK + 8 * ch)) for ch in range(3)], axis=-1)
    s = None
    if seg is not None:
        s = seg.copy()
        models = [cfg.get(k, 0) for k in ("seg_gauss", "seg_speckle", "seg_shot", "seg_salt_pepper")]
        if any(m > 0 for m in models):
            v = np.rint(_noisy(s.astype(np.float64), float(cfg["seg_max"]), *models, seed,
                               b + np.uint64(SEG_BLOCK))).astype(np.int64)
            s = np.where(s >= 0, v, -1).astype(seg.dtype)
        p = cfg.get("seg_dropout", 0)
        if p > 0:
            drop = _u_half_open(splitmix64(seed, b + np.uint64(SEG_DROPOUT))) < np.float64(np.float32(p))
            s[drop] = -1
    return d, c, s
