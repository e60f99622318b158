"""The benchmark workloads, named by what they are.

``seed = 190506228 + 1000 * workload_index + pair``, PCG64 streams.

=====================  =====================================================
name                   content
=====================  =====================================================
rigid256               1 pair 256x256, 3000 speckles, rigid (3.4, -2.7) px,
                       no noise; subset 21, step 10, search +-10 px
affine1024             1 pair 1024x1024, 40000 speckles, affine
                       exx=0.5 %, eyy=-0.2 %, 1 deg, t=(7.3, 4.1), noise 2;
                       subset 31, step 5, search +-20 px
sine2048x64            64 pairs 2048x2048, 160000 speckles each,
                       u=2 sin(2 pi y/128), v=1.5 cos(2 pi x/96) plus a
                       per-pair rigid offset U(-15, 15)^2; subset 41,
                       step 8, search +-24 px
mixed32                32 pairs: 8 each of 512^2, 1024^2, 2048^2, 4096^2,
                       0.04 speckles/px^2, random affine (|e|<=1 %,
                       |theta|<=2 deg, |t|<=5 px), noise U(1, 3), subset
                       from {15, 21, 31, 41, 51}, step floor(subset/3)
affine1024x8           8 pairs as affine1024 (deformation and noise),
                       subset 31, step 8, search +-20 px
tensile1024x16         17 frames 1024x1024 of one speckle pattern (40000
                       speckles, noise 2) under a growing tensile load:
                       frame k has exx = 0.05 % k, eyy = -0.015 % k and a
                       drift of (0.35, -0.1) px per frame; 16 consecutive
                       pairs (reference updated every frame); subset 31,
                       step 5, search +-12 px (a window of 25 pixels)
=====================  =====================================================
"""
from __future__ import annotations

import math

import numpy as np

from .speckle import Affine, Pair, Rigid, Sinusoidal, render_pair, render_sequence

SEED_BASE = 190506228

WORKLOADS = ("rigid256", "affine1024", "sine2048x64", "mixed32", "affine1024x8",
             "tensile1024x16")


def seed_of(workload_index: int, pair: int) -> int:
    return SEED_BASE + 1000 * workload_index + pair


def rigid256(pair: int = 0) -> Pair:
    d = Rigid(3.4, -2.7)
    f, g = render_pair(seed_of(0, pair), 256, 256, 3000, d, 0.0, pad=24.0)
    return Pair(f, g, d, subset=21, step=10, radius=10, meta={"workload": "rigid256"})


def _affine1024_map() -> Affine:
    return Affine(exx=0.005, eyy=-0.002, theta_deg=1.0, tx=7.3, ty=4.1,
                  cx=(1024 - 1) / 2.0, cy=(1024 - 1) / 2.0)


def affine1024(pair: int = 0) -> Pair:
    d = _affine1024_map()
    f, g = render_pair(seed_of(1, pair), 1024, 1024, 40000, d, 2.0, pad=40.0)
    return Pair(f, g, d, subset=31, step=5, radius=20, meta={"workload": "affine1024"})


def sine2048(pair: int) -> Pair:
    rng = np.random.Generator(np.random.PCG64(seed_of(2, 10_000 + pair)))
    t = rng.uniform(-15.0, 15.0, 2)
    d = Sinusoidal(tx=float(t[0]), ty=float(t[1]))
    f, g = render_pair(seed_of(2, pair), 2048, 2048, 160000, d, 0.0, pad=40.0)
    return Pair(f, g, d, subset=41, step=8, radius=24, meta={"workload": "sine2048x64"})


MIXED_SIZES = (512, 1024, 2048, 4096)
MIXED_SUBSETS = (15, 21, 31, 41, 51)


def mixed_params(pair: int) -> dict:
    """Per-pair parameters of the mixed-size batch (no pixels rendered)."""
    rng = np.random.Generator(np.random.PCG64(seed_of(3, 10_000 + pair)))
    size = MIXED_SIZES[pair // 8]
    exx, eyy = rng.uniform(-0.01, 0.01, 2)
    theta = rng.uniform(-2.0, 2.0)
    t = rng.uniform(-5.0, 5.0, 2)
    sigma = rng.uniform(1.0, 3.0)
    subset = int(MIXED_SUBSETS[rng.integers(0, len(MIXED_SUBSETS))])
    c = (size - 1) / 2.0
    d = Affine(float(exx), float(eyy), float(theta), float(t[0]), float(t[1]), c, c)
    # search radius: largest displacement component anywhere in the image, + 2
    xs = np.array([0.0, size - 1.0, 0.0, size - 1.0])
    ys = np.array([0.0, 0.0, size - 1.0, size - 1.0])
    u, _, _, v, _, _ = d.displacement(xs, ys)
    radius = int(math.ceil(max(np.abs(u).max(), np.abs(v).max()))) + 2
    return dict(size=size, deformation=d, sigma=float(sigma), subset=subset,
                step=subset // 3, radius=radius, n_speckles=int(round(0.04 * size * size)))


def mixed(pair: int) -> Pair:
    p = mixed_params(pair)
    f, g = render_pair(seed_of(3, pair), p["size"], p["size"], p["n_speckles"],
                       p["deformation"], p["sigma"], pad=p["radius"] + 20.0)
    return Pair(f, g, p["deformation"], subset=p["subset"], step=p["step"],
                radius=p["radius"], meta={"workload": "mixed32", "sigma": p["sigma"]})


def affine1024x8(pair: int) -> Pair:
    d = _affine1024_map()
    f, g = render_pair(seed_of(4, pair), 1024, 1024, 40000, d, 2.0, pad=40.0)
    return Pair(f, g, d, subset=31, step=8, radius=20, meta={"workload": "affine1024x8"})


def tensile_sequence(frames: int = 17, size: int = 1024, n_speckles: int = 40000,
                     noise: float = 2.0, seed_index: int = 5) -> dict:
    """Frames of the tensile sequence and its analysis parameters; frame k
    is the pattern under exx = 5e-4 k, eyy = -1.5e-4 k, t = (0.35 k, -0.1 k)
    about the image centre."""
    c = (size - 1) / 2.0
    maps = [None] + [Affine(5e-4 * k, -1.5e-4 * k, 0.0, 0.35 * k, -0.1 * k, c, c)
                     for k in range(1, frames)]
    imgs = render_sequence(seed_of(seed_index, 0), size, size, n_speckles, maps, noise,
                           pad=40.0)
    return dict(frames=imgs, maps=maps, subset=31, step=5, radius=12)


def tiny(seed: int, width: int = 24, height: int = 24, n_speckles: int = 40,
         deformation=None, noise: float = 0.0) -> tuple[np.ndarray, np.ndarray]:
    """Small pair for brute-force checks."""
    if deformation is None:
        deformation = Rigid(1.0, -2.0)
    return render_pair(seed, width, height, n_speckles, deformation, noise, pad=6.0)
