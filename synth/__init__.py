"""Seeded synthetic inputs for homogeneous diffusion inpainting.

This module is shared by the CPU oracle's tests, the GPU parity tests and the
benchmark.  It holds none of the solver's arithmetic: it only draws images and
masks.  The paper evaluates on twelve 4K photographs with optimized masks
(Section 5.1); neither is available, so these generators stand in for them with
the same sizes (up to 3840x2160, 3 channels) and the same mask densities
(0.5 % to 10 %, Section 5.2).

Image model (per channel k, seed + k): the sum of four plane sinusoids with
random direction, wavelength, amplitude and phase, then three disks of constant
value painted over it, then an affine map onto [0, 255].  Masks are binary
(Section 2.2) and shared by all channels: uniform Bernoulli(d), or exactly
round(d * N) pixels drawn without replacement with probability proportional to
|LoG_sigma=2(f)| summed over channels plus a small floor (edge-clustered).
Every mask holds at least one pixel.

Video (a stand-in for image sequences, which the paper does not test): a
static background frame with one disk of constant value per channel moving
along a straight line, and one mask for the whole sequence, drawn on the first
frame (a fixed sampling pattern).
"""
from __future__ import annotations

import numpy as np

__all__ = ["image", "mask_uniform", "mask_edge", "make_case", "make_video"]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed) & 0xFFFFFFFFFFFFFFFF))


def image(width: int, height: int, channels: int, seed: int) -> np.ndarray:
    """Planar float32 image [channels][height][width] with values in [0, 255]."""
    out = np.empty((channels, height, width), dtype=np.float32)
    m = max(1, min(width, height))
    ys = np.arange(height, dtype=np.float64)[:, None]
    xs = np.arange(width, dtype=np.float64)[None, :]
    for k in range(channels):
        g = _rng(seed + k)
        field = np.zeros((height, width), dtype=np.float64)
        for _ in range(4):
            theta = g.uniform(0.0, np.pi)
            lam = g.uniform(m / 32.0, m / 2.0)
            amp = g.uniform(0.5, 1.0)
            phi = g.uniform(0.0, 2.0 * np.pi)
            proj = np.cos(theta) * xs + np.sin(theta) * ys
            field += amp * np.sin(2.0 * np.pi * proj / lam + phi)
        lo, hi = float(field.min()), float(field.max())
        for _ in range(3):
            cx = g.uniform(0.0, width)
            cy = g.uniform(0.0, height)
            rad = g.uniform(0.03, 0.15) * m
            val = g.uniform(lo, hi)
            inside = (xs - cx) ** 2 + (ys - cy) ** 2 <= rad * rad
            field = np.where(inside, val, field)
        lo, hi = float(field.min()), float(field.max())
        if hi > lo:
            field = (field - lo) * (255.0 / (hi - lo))
        else:
            field = np.zeros_like(field)
        out[k] = field.astype(np.float32)
    return out


def _force_one(mask: np.ndarray, g: np.random.Generator) -> np.ndarray:
    if not mask.any():
        idx = int(g.integers(0, mask.size))
        mask.reshape(-1)[idx] = 1
    return mask


def mask_uniform(width: int, height: int, density: float, seed: int) -> np.ndarray:
    """uint8 [height][width]: each pixel known with probability `density`."""
    g = _rng(seed ^ 0x5A5A5A5A)
    mask = (g.random((height, width)) < density).astype(np.uint8)
    return _force_one(mask, g)


def _log_magnitude(f: np.ndarray) -> np.ndarray:
    from scipy import ndimage

    acc = np.zeros(f.shape[1:], dtype=np.float64)
    for k in range(f.shape[0]):
        acc += np.abs(ndimage.gaussian_laplace(f[k].astype(np.float64), sigma=2.0,
                                               mode="reflect"))
    return acc


def mask_edge(f: np.ndarray, density: float, seed: int) -> np.ndarray:
    """uint8 mask with exactly round(density*N) pixels (at least one), drawn
    without replacement with weights |LoG(f)| + 1e-3*mean (Efraimidis-Spirakis
    keys log(U)/w, largest keys win)."""
    _, height, width = f.shape
    n = height * width
    k = int(round(density * n))
    k = min(max(k, 1), n)
    wgt = _log_magnitude(f).reshape(-1)
    mean = float(wgt.mean())
    wgt = wgt + (1e-3 * mean if mean > 0 else 1.0)
    g = _rng(seed ^ 0x0EDC0EDC)
    keys = np.log(g.random(n)) / wgt
    chosen = np.argpartition(keys, n - k)[n - k:]
    mask = np.zeros(n, dtype=np.uint8)
    mask[chosen] = 1
    return mask.reshape(height, width)


def make_case(width: int, height: int, channels: int, density: float, kind: str,
              seed: int):
    """(f, c) for one synthetic case; kind is 'uniform' or 'edge'."""
    f = image(width, height, channels, seed)
    if kind == "uniform":
        c = mask_uniform(width, height, density, seed)
    elif kind == "edge":
        c = mask_edge(f, density, seed)
    else:
        raise ValueError(f"unknown mask kind {kind!r}")
    return f, c


def make_video(width: int, height: int, channels: int, density: float, kind: str, seed: int,
               frames: int, speed: float = 2.0):
    """([f_0, ..., f_{frames-1}], c): the background of make_case(seed) with a
    disk of radius min(w, h)/10 crossing it at `speed` pixels per frame; c is
    drawn on frame 0 and shared by all frames."""
    base = image(width, height, channels, seed)
    g = _rng(seed + 7919)
    m = max(1, min(width, height))
    rad = m / 10.0
    y0, x0 = g.uniform(0.3, 0.7) * height, g.uniform(0.2, 0.4) * width
    ang = g.uniform(-0.5, 0.5)
    vals = g.uniform(0.0, 255.0, size=channels)
    ys = np.arange(height, dtype=np.float64)[:, None]
    xs = np.arange(width, dtype=np.float64)[None, :]
    seq = []
    for t in range(frames):
        cx = x0 + t * speed * np.cos(ang)
        cy = y0 + t * speed * np.sin(ang)
        inside = (xs - cx) ** 2 + (ys - cy) ** 2 <= rad * rad
        f = base.copy()
        for k in range(channels):
            f[k][inside] = vals[k]
        seq.append(f)
    if kind == "uniform":
        c = mask_uniform(width, height, density, seed)
    elif kind == "edge":
        c = mask_edge(seq[0], density, seed)
    else:
        raise ValueError(f"unknown mask kind {kind!r}")
    return seq, c
