"""Seeded synthetic images for the Gauss-polynomial bilateral filter workloads.

This module only draws inputs; it holds none of the filter's arithmetic.  Both
the CUDA path's tests/benchmark and the FP64 oracle's tests take their images
from here, so the two sides always see the same pixels.

Recipe (one numpy PCG64 generator per image, seeded):
  1. background level ~ U[0, 255]
  2. n_rect axis-aligned rectangles painted in order; per axis the two corners
     are two sorted uniform integers in [0, size]; level ~ U[0, 255]
     (for multi-plane images the geometry is shared and each plane draws its
     own level)
  3. optional ramp: ramp_amp * sin(2 pi (0.75 x / W + 0.5 y / H) + phi),
     phi ~ U[0, 2 pi)
  4. additive N(0, noise_std^2) per pixel
  5. clip to [0, 255]
  6. stored as float32 (not quantised)

The paper's own test image (the 256x256 Peppers picture used in its Table 1
and Fig. 4) is not available; these piecewise-constant-plus-noise images stand
in for it and for the larger workloads.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 150500077  # arXiv 1505.00077


def seed_for(family: int, index: int = 0) -> int:
    """Seed of image `index` of a workload family (a small integer per workload)."""
    return SEED_BASE + 1000 * int(family) + int(index)


def make_image(H: int, W: int, n_rect: int, noise_std: float, ramp_amp: float = 0.0,
               seed: int = 0, planes: int = 1) -> np.ndarray:
    """Return a float32 array [planes, H, W] (or [H, W] when planes == 1)."""
    rng = np.random.default_rng(seed)
    img = np.empty((planes, H, W), np.float64)
    for c in range(planes):
        img[c].fill(rng.uniform(0.0, 255.0))
    for _ in range(n_rect):
        y0, y1 = np.sort(rng.integers(0, H + 1, size=2))
        x0, x1 = np.sort(rng.integers(0, W + 1, size=2))
        for c in range(planes):
            img[c, y0:y1, x0:x1] = rng.uniform(0.0, 255.0)
    if ramp_amp:
        phi = rng.uniform(0.0, 2.0 * math.pi)
        yy = np.arange(H, dtype=np.float64)[:, None] / H
        xx = np.arange(W, dtype=np.float64)[None, :] / W
        img += ramp_amp * np.sin(2.0 * math.pi * (0.75 * xx + 0.5 * yy) + phi)[None]
    if noise_std:
        img += rng.normal(0.0, noise_std, size=img.shape)
    np.clip(img, 0.0, 255.0, out=img)
    out = img.astype(np.float32)
    return out[0] if planes == 1 else out


# ---------------------------------------------------------------- workloads


@dataclass(frozen=True)
class PlaneSpec:
    H: int
    W: int
    sigma_s: float
    sigma_r: float
    order: int
    seed: int
    n_rect: int
    noise_std: float
    ramp_amp: float = 0.0


def rects256_image() -> np.ndarray:
    """256x256, 16 rectangles, noise std 10 (sigma_s 3, sigma_r 30)."""
    return make_image(256, 256, 16, 10.0, 0.0, seed_for(1))


def rects_ramp1024_image() -> np.ndarray:
    """1024x1024, 64 rectangles + sinusoidal ramp of amplitude 60, noise std 10."""
    return make_image(1024, 1024, 64, 10.0, 60.0, seed_for(2))


def rects4096_image() -> np.ndarray:
    """4096x4096 (16.7 Mpx), 512 rectangles, noise std 15 (sigma_s 10, sigma_r 20)."""
    return make_image(4096, 4096, 512, 15.0, 0.0, seed_for(3))


def uneven_batch_specs(n_images: int = 64, order: int = 20):
    """Batched workload: n_images images, sides ~ U{256..2048} independently,
    3 planes each; per image sigma_s ~ logU[1, 16], sigma_r ~ logU[10, 60];
    16 rectangles per 256^2 of area, noise std 10.  Returns a list of
    (image_index, H, W, sigma_s, sigma_r, n_rect, seed)."""
    rng = np.random.default_rng(seed_for(4, 999))
    out = []
    for i in range(n_images):
        H = int(rng.integers(256, 2049))
        W = int(rng.integers(256, 2049))
        ss = float(math.exp(rng.uniform(math.log(1.0), math.log(16.0))))
        sr = float(math.exp(rng.uniform(math.log(10.0), math.log(60.0))))
        n_rect = max(1, int(round(16 * H * W / (256 * 256))))
        out.append((i, H, W, ss, sr, n_rect, seed_for(4, i)))
    return out


def uneven_batch_image(spec) -> np.ndarray:
    _, H, W, _, _, n_rect, seed = spec
    return make_image(H, W, n_rect, 10.0, 0.0, seed, planes=3)


def batch512(batch: int = 16) -> np.ndarray:
    """[batch, 1, 512, 512], 32 rectangles, noise std 10 (sigma_s 5, sigma_r 25)."""
    return np.stack([make_image(512, 512, 32, 10.0, 0.0, seed_for(5, i))[None] for i in range(batch)])
