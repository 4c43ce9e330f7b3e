"""Seeded synthetic inputs for the adaptive bilateral filter.

This module holds no arithmetic of the filter itself: it only draws the
8-bit image f, the range-kernel centre theta(i) and the range-kernel width
sigma(i) that the filter consumes (Sec. I-A, Eqs. (1)-(3) of the paper:
an 8-bit image, a per-pixel centre and a per-pixel width).  Both the CUDA
path and the CPU oracle are fed from here; neither imports the other.

The paper's own test images (natural photographs of 512x512 to 1066x584)
are not available, so a seeded stand-in with the same structure is drawn:
smooth shading (Gaussian blobs), a few sharp step edges and sensor-like
Gaussian noise, clipped to the 8-bit range.

Recipe (all draws from ``numpy.random.default_rng(seed)``, in this order):

* ``n_blobs`` Gaussian blobs ``A_b exp(-|x-c_b|^2 / (2 s_b^2))`` with centre
  ``c_b`` uniform over the image, amplitude ``A_b ~ U[0, 200]`` and width
  ``s_b ~ U[0.1, 0.6] * sqrt(H W / n_blobs)`` (so the blob density does not
  depend on the image size; at 256x256 with 20 blobs this is 5.7..34 px).
  Each blob is evaluated within 6 s_b of its centre.
* 4 step edges: a line through a uniform point at a uniform angle; one side
  of it is raised by ``h ~ U[60, 120]`` times a random sign.
* a base level of 64 gray levels, then i.i.d. ``N(0, noise_sigma^2)`` noise;
  clip to [0, 255]; round half to even; cast to uint8.
* smooth fields (theta offset zeta, sigma): an 8x8 grid of ``U[lo, hi]``
  values upsampled bilinearly (corner-aligned) to H x W, float32.

Colour images (``make_rgb``, interleaved H x W x 3) follow the same recipe
with one geometry for the three channels: each blob draws its centre and
width once and an amplitude per channel, each edge its line once and a
height per channel (one sign), and the noise is independent per channel.

The spatial kernel is an input too: ``gaussian_taps(rho)`` gives the integer
taps of a Gaussian of width rho on the paper's window [-3 rho, 3 rho]
(Eq. (4)), and ``random_taps`` draws arbitrary (asymmetric) taps for tests.
"""
from __future__ import annotations

import numpy as np

__all__ = ["make_image", "make_rgb", "smooth_field", "make_inputs", "config_seed", "gaussian_taps",
           "random_taps"]


def config_seed(config: int, index: int) -> int:
    """Seed of image ``index`` of workload ``config`` (1000 * config + index)."""
    return 1000 * int(config) + int(index)


def make_image(H: int, W: int, n_blobs: int, rng: np.random.Generator,
               noise_sigma: float = 10.0, n_edges: int = 4) -> np.ndarray:
    """Draw one H x W uint8 image (blobs + step edges + noise), see module doc."""
    img = np.full((H, W), 64.0, dtype=np.float64)
    scale = np.sqrt(H * W / max(n_blobs, 1))
    for _ in range(n_blobs):
        cy = rng.uniform(0.0, H)
        cx = rng.uniform(0.0, W)
        s = rng.uniform(0.1, 0.6) * scale
        a = rng.uniform(0.0, 200.0)
        r = int(np.ceil(6.0 * s))
        y0, y1 = max(0, int(cy) - r), min(H, int(cy) + r + 1)
        x0, x1 = max(0, int(cx) - r), min(W, int(cx) + r + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        dy = (np.arange(y0, y1, dtype=np.float64) - cy)[:, None]
        dx = (np.arange(x0, x1, dtype=np.float64) - cx)[None, :]
        img[y0:y1, x0:x1] += a * np.exp(-(dy * dy + dx * dx) / (2.0 * s * s))
    yy = np.arange(H, dtype=np.float64)[:, None]
    xx = np.arange(W, dtype=np.float64)[None, :]
    for _ in range(n_edges):
        py = rng.uniform(0.0, H)
        px = rng.uniform(0.0, W)
        ang = rng.uniform(0.0, 2.0 * np.pi)
        h = rng.uniform(60.0, 120.0) * (1.0 if rng.uniform() < 0.5 else -1.0)
        side = ((xx - px) * np.cos(ang) + (yy - py) * np.sin(ang)) > 0.0
        img += h * side
    img += rng.normal(0.0, noise_sigma, size=(H, W))
    return np.rint(np.clip(img, 0.0, 255.0)).astype(np.uint8)


def make_rgb(H: int, W: int, seed: int, n_blobs: int = 20, noise_sigma: float = 10.0,
             n_edges: int = 4) -> np.ndarray:
    """Draw one H x W x 3 interleaved uint8 colour image, see module doc."""
    rng = np.random.default_rng(seed)
    img = np.full((H, W, 3), 64.0, dtype=np.float64)
    scale = np.sqrt(H * W / max(n_blobs, 1))
    for _ in range(n_blobs):
        cy = rng.uniform(0.0, H)
        cx = rng.uniform(0.0, W)
        s = rng.uniform(0.1, 0.6) * scale
        a = rng.uniform(0.0, 200.0, size=3)
        r = int(np.ceil(6.0 * s))
        y0, y1 = max(0, int(cy) - r), min(H, int(cy) + r + 1)
        x0, x1 = max(0, int(cx) - r), min(W, int(cx) + r + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        dy = (np.arange(y0, y1, dtype=np.float64) - cy)[:, None]
        dx = (np.arange(x0, x1, dtype=np.float64) - cx)[None, :]
        img[y0:y1, x0:x1] += np.exp(-(dy * dy + dx * dx) / (2.0 * s * s))[:, :, None] * a
    yy = np.arange(H, dtype=np.float64)[:, None]
    xx = np.arange(W, dtype=np.float64)[None, :]
    for _ in range(n_edges):
        py = rng.uniform(0.0, H)
        px = rng.uniform(0.0, W)
        ang = rng.uniform(0.0, 2.0 * np.pi)
        h = rng.uniform(60.0, 120.0, size=3) * (1.0 if rng.uniform() < 0.5 else -1.0)
        side = ((xx - px) * np.cos(ang) + (yy - py) * np.sin(ang)) > 0.0
        img += side[:, :, None] * h
    img += rng.normal(0.0, noise_sigma, size=(H, W, 3))
    return np.ascontiguousarray(np.rint(np.clip(img, 0.0, 255.0)).astype(np.uint8))


def smooth_field(H: int, W: int, lo: float, hi: float,
                 rng: np.random.Generator, grid: int = 8) -> np.ndarray:
    """Bilinear (corner-aligned) upsampling of a grid x grid U[lo, hi] array."""
    g = rng.uniform(lo, hi, size=(grid, grid))
    ys = np.linspace(0.0, grid - 1.0, H) if H > 1 else np.zeros(1)
    xs = np.linspace(0.0, grid - 1.0, W) if W > 1 else np.zeros(1)
    y0 = np.minimum(np.floor(ys).astype(np.int64), grid - 2)
    x0 = np.minimum(np.floor(xs).astype(np.int64), grid - 2)
    fy = (ys - y0)[:, None]
    fx = (xs - x0)[None, :]
    g00 = g[y0][:, x0]
    g01 = g[y0][:, x0 + 1]
    g10 = g[y0 + 1][:, x0]
    g11 = g[y0 + 1][:, x0 + 1]
    out = (g00 * (1 - fy) * (1 - fx) + g01 * (1 - fy) * fx
           + g10 * fy * (1 - fx) + g11 * fy * fx)
    return np.clip(out, lo, hi).astype(np.float32)


def make_inputs(H: int, W: int, seed: int, n_blobs: int = 20,
                sigma_range=(10.0, 40.0), zeta_range=None,
                noise_sigma: float = 10.0):
    """Return ``(f, theta, sigma)``: uint8 image and float32 centre/width maps.

    ``theta = f`` (classical centre) when ``zeta_range`` is None, else
    ``theta = f + zeta`` with ``zeta`` a smooth field in ``zeta_range``.
    All three arrays are C-contiguous, shape (H, W).
    """
    rng = np.random.default_rng(seed)
    f = make_image(H, W, n_blobs, rng, noise_sigma=noise_sigma)
    if zeta_range is None:
        theta = f.astype(np.float32)
    else:
        zeta = smooth_field(H, W, zeta_range[0], zeta_range[1], rng)
        theta = (f.astype(np.float32) + zeta).astype(np.float32)
    sigma = smooth_field(H, W, sigma_range[0], sigma_range[1], rng)
    return (np.ascontiguousarray(f), np.ascontiguousarray(theta),
            np.ascontiguousarray(sigma))


def gaussian_taps(rho: float, peak: int = 1024) -> np.ndarray:
    """Integer taps of the Gaussian spatial kernel of Eq. (4), one axis.

    ``r = ceil(3 rho)`` (window [-3 rho, 3 rho]) and ``g[t] = floor(peak
    exp(-(t - r)^2 / (2 rho^2)) + 1/2)`` for t = 0..2r, uint32.  With
    peak = 1024 and rho <= 40/3 (r <= 40) the taps sum to at most 34,300.
    The 2-D kernel is g[ty + r] g[tx + r].
    """
    if not (rho > 0):
        raise ValueError("rho must be positive")
    r = int(np.ceil(3.0 * rho))
    t = np.arange(-r, r + 1, dtype=np.float64)
    return np.floor(peak * np.exp(-t * t / (2.0 * rho * rho)) + 0.5).astype(np.uint32)


def random_taps(r: int, rng: np.random.Generator, hi: int = 1000) -> np.ndarray:
    """2r+1 arbitrary taps in [0, hi] with a non-zero centre (uint32)."""
    g = rng.integers(0, hi + 1, size=2 * r + 1).astype(np.uint32)
    g[r] = max(int(g[r]), 1)
    return g
