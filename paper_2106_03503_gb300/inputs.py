"""Seeded synthetic inputs for the distance-transform workloads.

This module holds no distance-transform arithmetic: it only draws masks.  Both
the CUDA path's tests and benchmark and the CPU oracle take their inputs from
here, so that the two sides see identical bytes.  Everything is numpy
(``default_rng(seed)``), deterministic for a given seed.

Workloads (sizes and value distributions of the distance-transform use cases
the paper describes in Sec. 1.1; the paper ships no data):
  * ``bernoulli_mask``      isolated object points (Fig. 2, "30 separate object
                            points"), each pixel an object with probability p;
  * ``discs_mask``          many filled discs (blob images as in Fig. 3),
                            clipped at the image border;
  * ``smoothed_noise_volume`` 3-D blobs: white Gaussian noise smoothed with an
                            isotropic Gaussian, thresholded at 0;
  * ``batch_masks``         many 2-D masks of uneven sizes and densities;
  * ``serving_jobs``        a Poisson stream of mixed 2-D / 3-D jobs.
"""
from __future__ import annotations

import math

import numpy as np


def bernoulli_mask(shape, p: float, seed: int) -> np.ndarray:
    """uint8 mask, each pixel 1 with probability p (independently)."""
    rng = np.random.default_rng(seed)
    return (rng.random(shape) < p).astype(np.uint8)


def discs_mask(H: int, W: int, n_discs: int, r_min: int, r_max: int, seed: int) -> np.ndarray:
    """Union of n_discs filled discs: integer centres uniform over the image,
    integer radii uniform in [r_min, r_max]; pixel (y, x) is inside when
    (x - cx)^2 + (y - cy)^2 <= r^2.  Discs are clipped at the border."""
    rng = np.random.default_rng(seed)
    cy = rng.integers(0, H, size=n_discs)
    cx = rng.integers(0, W, size=n_discs)
    r = rng.integers(r_min, r_max + 1, size=n_discs)
    m = np.zeros((H, W), dtype=np.uint8)
    for y0, x0, rr in zip(cy.tolist(), cx.tolist(), r.tolist()):
        ya, yb = max(0, y0 - rr), min(H, y0 + rr + 1)
        xa, xb = max(0, x0 - rr), min(W, x0 + rr + 1)
        yy = np.arange(ya, yb)[:, None] - y0
        xx = np.arange(xa, xb)[None, :] - x0
        m[ya:yb, xa:xb] |= ((yy * yy + xx * xx) <= rr * rr).astype(np.uint8)
    return m


def smoothed_noise_volume(shape, sigma: float, seed: int, threshold: float = 0.0) -> np.ndarray:
    """float32 N(0,1) noise smoothed by an isotropic Gaussian of std sigma
    (periodic boundary, applied as the transfer function exp(-2 pi^2 sigma^2
    |f|^2) in the Fourier domain), then mask = smoothed > threshold."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(shape, dtype=np.float32)
    try:
        import scipy.fft as sfft
        spec = sfft.rfftn(noise, workers=-1)
    except Exception:  # pragma: no cover - scipy is present on both machines
        sfft = None
        spec = np.fft.rfftn(noise)
    transfer = np.ones(spec.shape, dtype=np.float32)
    for axis, n in enumerate(shape):
        if axis == len(shape) - 1:
            f = np.fft.rfftfreq(n).astype(np.float32)
        else:
            f = np.fft.fftfreq(n).astype(np.float32)
        g = np.exp(-2.0 * math.pi ** 2 * sigma ** 2 * f * f).astype(np.float32)
        sh = [1] * len(shape)
        sh[axis] = g.shape[0]
        transfer = transfer * g.reshape(sh)
    spec *= transfer
    if sfft is not None:
        smooth = sfft.irfftn(spec, s=shape, workers=-1)
    else:  # pragma: no cover
        smooth = np.fft.irfftn(spec, s=shape)
    return (smooth > threshold).astype(np.uint8)


def batch_masks(n: int, side_lo: int, side_hi: int, p_lo: float, p_hi: float, seed: int):
    """n 2-D Bernoulli masks: H and W uniform integers in [side_lo, side_hi],
    density log-uniform in [p_lo, p_hi].  Returns a list of uint8 arrays."""
    rng = np.random.default_rng(seed)
    Hs = rng.integers(side_lo, side_hi + 1, size=n)
    Ws = rng.integers(side_lo, side_hi + 1, size=n)
    ps = np.exp(rng.uniform(math.log(p_lo), math.log(p_hi), size=n))
    out = []
    for h, w, p in zip(Hs.tolist(), Ws.tolist(), ps.tolist()):
        out.append((rng.random((h, w)) < p).astype(np.uint8))
    return out


def serving_jobs(n: int, seed: int, frac_2d: float = 0.8, side2d=(128, 4096), side3d=(64, 256),
                 p_lo: float = 0.001, p_hi: float = 0.1, sigma3d: float = 4.0):
    """Job descriptions for a serving run (masks are drawn lazily by
    ``draw_job`` so that large streams need not be held in memory).

    Each job is 2-D with probability frac_2d (square side uniform in side2d,
    Bernoulli density log-uniform in [p_lo, p_hi]) and otherwise 3-D (cube side
    uniform in side3d, smoothed noise sigma3d thresholded at 0)."""
    rng = np.random.default_rng(seed)
    jobs = []
    for t in range(n):
        if rng.random() < frac_2d:
            s = int(rng.integers(side2d[0], side2d[1] + 1))
            p = float(np.exp(rng.uniform(math.log(p_lo), math.log(p_hi))))
            jobs.append({"ndim": 2, "shape": (s, s), "p": p, "seed": seed * 1_000_003 + t})
        else:
            s = int(rng.integers(side3d[0], side3d[1] + 1))
            jobs.append({"ndim": 3, "shape": (s, s, s), "sigma": sigma3d, "seed": seed * 1_000_003 + t})
    return jobs


def draw_job(job) -> np.ndarray:
    """Materialise the mask of one ``serving_jobs`` entry."""
    if job["ndim"] == 2:
        return bernoulli_mask(job["shape"], job["p"], job["seed"])
    return smoothed_noise_volume(job["shape"], job["sigma"], job["seed"])


# Named workloads ------------------------------------------------------------

def points_512(seed: int = 1) -> np.ndarray:
    """512 x 512, each pixel an object with probability 0.01."""
    return bernoulli_mask((512, 512), 0.01, seed)


def discs_8192(seed: int = 2) -> np.ndarray:
    """8192 x 8192, union of 2000 discs with radii 5..60 (about 11.6 % object)."""
    return discs_mask(8192, 8192, 2000, 5, 60, seed)


def blobs_512cube(seed: int = 3) -> np.ndarray:
    """512^3 smoothed Gaussian noise (sigma 4) thresholded at 0 (about 50 %)."""
    return smoothed_noise_volume((512, 512, 512), 4.0, seed)


def batch_4096(seed: int = 4, n: int = 4096):
    """4096 masks, sides uniform in [64, 1024], density log-uniform [0.001, 0.1]."""
    return batch_masks(n, 64, 1024, 0.001, 0.1, seed)
