"""Seeded synthetic images and additive white Gaussian noise.

This module holds no denoising arithmetic.  It only draws the inputs that
both the GPU path and the FP64 oracle consume, so that the two sides see the
same numbers.

Observation model (Eq. 1): y = x + n, n ~ N(0, sigma^2) i.i.d. per pixel,
on a 0..255 scale, not clipped.

Clean-scene recipe (stand-in for the paper's natural-image test sets, which
are not available here):
  * 8 Voronoi cells, each a linear ramp a + b*(x - sx) + c*(y - sy) with
    a ~ U[30, 225] and slopes b, c ~ U[-0.15, 0.15] per pixel;
  * 3 of the cells carry an oriented sinusoidal grating, amplitude
    U[20, 60], orientation U[0, pi), period U[4, 16] px, phase U[0, 2 pi);
  * one axis-aligned rectangle of about 1/8 of the image area is filled with
    a 16x16 tile of U[0, 255] values repeated with period 16 from the
    rectangle's top-left corner;
  * the result is clipped to [0, 255].
RGB scenes reuse the geometry (cells, grating directions, tile placement)
and draw independent per-channel levels and amplitudes.
"""
from __future__ import annotations

import numpy as np

NOISE_SEED_MUL = 1_000_003


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def make_image_with_meta(seed: int, H: int, W: int, C: int = 1):
    """Clean scene float32 [C, H, W] in [0, 255] and the tile rectangle (ty, tx, th, tw)."""
    if H <= 0 or W <= 0 or C not in (1, 3):
        raise ValueError("make_image: need H, W > 0 and C in {1, 3}")
    rng = _rng(seed)
    n_cells = 8
    sx = rng.uniform(0, W, n_cells)
    sy = rng.uniform(0, H, n_cells)
    slope_b = rng.uniform(-0.15, 0.15, n_cells)
    slope_c = rng.uniform(-0.15, 0.15, n_cells)
    level = rng.uniform(30, 225, (C, n_cells))
    g_cells = rng.choice(n_cells, size=3, replace=False)
    g_theta = rng.uniform(0, np.pi, 3)
    g_period = rng.uniform(4, 16, 3)
    g_phase = rng.uniform(0, 2 * np.pi, 3)
    g_amp = rng.uniform(20, 60, (C, 3))
    th = max(1, int(round(H / np.sqrt(8.0))))
    tw = max(1, int(round(W / np.sqrt(8.0))))
    ty = int(rng.integers(0, H - th + 1))
    tx = int(rng.integers(0, W - tw + 1))
    tile = rng.uniform(0, 255, (C, 16, 16))

    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    cell = np.zeros((H, W), np.int64)
    best = np.full((H, W), np.inf)
    for k in range(n_cells):
        d2 = (xx - sx[k]) ** 2 + (yy - sy[k]) ** 2
        m = d2 < best
        cell[m] = k
        best[m] = d2[m]
    out = np.empty((C, H, W), np.float64)
    ry = (np.arange(th) % 16)[:, None]
    rx = (np.arange(tw) % 16)[None, :]
    for c in range(C):
        img = (level[c][cell] + slope_b[cell] * (xx - sx[cell])
               + slope_c[cell] * (yy - sy[cell]))
        for g in range(3):
            m = cell == g_cells[g]
            u = xx * np.cos(g_theta[g]) + yy * np.sin(g_theta[g])
            img = img + m * g_amp[c, g] * np.sin(2 * np.pi * u / g_period[g] + g_phase[g])
        img[ty:ty + th, tx:tx + tw] = tile[c][ry, rx]
        out[c] = img
    return np.clip(out, 0.0, 255.0).astype(np.float32), (ty, tx, th, tw)


def make_image(seed: int, H: int, W: int, C: int = 1) -> np.ndarray:
    """Clean scene, float32 [C, H, W] in [0, 255]."""
    return make_image_with_meta(seed, H, W, C)[0]


def noise_seed(img_seed: int, sigma: float) -> int:
    return NOISE_SEED_MUL * int(img_seed) + int(round(float(sigma) * 1000.0))


def add_awgn(clean: np.ndarray, sigma: float, img_seed: int) -> np.ndarray:
    """y = x + n (Eq. 1); n ~ N(0, sigma^2), float32, not clipped."""
    rng = _rng(noise_seed(img_seed, sigma))
    n = rng.standard_normal(clean.shape) * float(sigma)
    return (clean.astype(np.float64) + n).astype(np.float32)


def make_batch(seeds, H: int, W: int, sigma, C: int = 1):
    """(clean, noisy) float32 [B, C, H, W]; sigma is a scalar or one per image."""
    seeds = list(seeds)
    sig = np.broadcast_to(np.asarray(sigma, np.float64), (len(seeds),))
    clean = np.stack([make_image(s, H, W, C) for s in seeds])
    noisy = np.stack([add_awgn(clean[i], sig[i], s) for i, s in enumerate(seeds)])
    return clean, noisy


def he_normal_weights(seed: int, layers: int = 10, width: int = 32, cin: int = 2, cout: int = 1):
    """He-normal initial weights for the residual CNN, zero biases.

    Returns a list of (W [Cout, 3, 3, Cin] float32, b [Cout] float32)."""
    rng = _rng(seed)
    out = []
    for l in range(layers):
        ci = cin if l == 0 else width
        co = cout if l == layers - 1 else width
        std = np.sqrt(2.0 / (9 * ci))
        w = (rng.standard_normal((co, 3, 3, ci)) * std).astype(np.float32)
        out.append((w, np.zeros(co, np.float32)))
    return out
