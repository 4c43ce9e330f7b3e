"""Pins of the oracle's colour functions (Sec. IV-C; no GPU).

Colour images are filtered channel by channel, and the texture width map is
computed on a gray version of the image.  The gray version is read as the
BT.601 luma rounded half up, in integers.  Pins:
  * luma of the primaries and of white equals the textbook 8-bit values
    (76, 150, 29, 255), and a gray pixel (v, v, v) maps to v;
  * luma is within 1/2 of 0.299 R + 0.587 G + 0.114 B (exact rationals) on
    every one of a random sample, and is monotone in each channel;
  * a gray image replicated into three channels gives, in every channel,
    the gray filter and the gray texture pipeline (both pinned elsewhere);
  * constant colour images pass unchanged;
  * the colour texture pipeline is the composition the docstring states.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1811_02308_gb300 import synth


def lq_for(taps, lap_sat):
    return int(math.floor(lap_sat * float(int(taps.sum())) ** 2 + 0.5))


def test_luma_of_primaries_white_and_grays(oracle_mod):
    px = np.array([[[255, 0, 0], [0, 255, 0], [0, 0, 255], [255, 255, 255], [0, 0, 0]]], np.uint8)
    assert oracle_mod.luma(px).tolist() == [[76, 150, 29, 255, 0]]
    v = np.arange(256, dtype=np.uint8)
    grays = np.stack([v, v, v], axis=-1)[None]
    assert np.array_equal(oracle_mod.luma(grays)[0], v)


def test_luma_rounds_the_weighted_sum(oracle_mod):
    rng = np.random.default_rng(5)
    x = rng.integers(0, 256, size=(1, 4000, 3), dtype=np.uint8)
    y = oracle_mod.luma(x)[0]
    wts = (Fraction(299, 1000), Fraction(587, 1000), Fraction(114, 1000))
    for (r, g, b), yy in zip(x[0].tolist(), y.tolist()):
        exact = wts[0] * r + wts[1] * g + wts[2] * b
        assert abs(exact - yy) <= Fraction(1, 2)
        if exact - math.floor(exact) == Fraction(1, 2):
            assert yy == math.floor(exact) + 1          # half rounds up
    for c in range(3):                                   # monotone per channel
        up = x.astype(np.int64)
        up[..., c] = np.minimum(up[..., c] + 1, 255)
        assert np.all(oracle_mod.luma(up.astype(np.uint8)) >= y)


def test_filter_rgb_on_replicated_gray_is_the_gray_filter(oracle_mod):
    f, th, sg = synth.make_inputs(18, 23, 4, n_blobs=6, zeta_range=(-10.0, 10.0))
    rgb = np.stack([f, f, f], axis=-1)
    ref, _ = oracle_mod.fabf(f, th, sg, 3, 5)
    got = oracle_mod.filter_rgb(rgb, np.stack([th, th, th], axis=-1), sg, 3, 5)
    for c in range(3):
        assert np.array_equal(got[..., c], ref)
    ref0, _ = oracle_mod.fabf(f, f.astype(np.float32), sg, 3, 5)
    got0 = oracle_mod.filter_rgb(rgb, None, sg, 3, 5)
    for c in range(3):
        assert np.array_equal(got0[..., c], ref0)


def test_filter_rgb_channels_are_independent(oracle_mod):
    # channel c of the output depends on channel c of the input (and theta)
    # only: changing the other channels leaves it unchanged
    rgb = synth.make_rgb(15, 17, 8, n_blobs=5)
    _, _, sg = synth.make_inputs(15, 17, 9)
    a = oracle_mod.filter_rgb(rgb, None, sg, 2, 4)
    other = rgb.copy()
    other[..., 1] = 255 - other[..., 1]
    other[..., 2] = other[..., 2] // 2
    b = oracle_mod.filter_rgb(other, None, sg, 2, 4)
    assert np.array_equal(a[..., 0], b[..., 0])
    assert not np.array_equal(a[..., 1], b[..., 1])


def test_texture_rgb_on_replicated_gray_is_the_gray_pipeline(oracle_mod):
    f, _, _ = synth.make_inputs(16, 21, 12, n_blobs=6)
    rgb = np.stack([f, f, f], axis=-1)
    taps = synth.gaussian_taps(1.0)
    Lq = lq_for(taps, 10.0)
    ref, _ = oracle_mod.texture_filter(f, 3, 4, 2, 1.0, 8.0, 5.0, 60.0, taps, Lq, 10.0, 40.0)
    got = oracle_mod.texture_filter_rgb(rgb, 3, 4, 2, 1.0, 8.0, 5.0, 60.0, taps, Lq, 10.0, 40.0)
    for c in range(3):
        assert np.array_equal(got[..., c], ref)


def test_texture_rgb_keeps_constant_colour(oracle_mod):
    rgb = np.empty((9, 11, 3), np.uint8)
    rgb[...] = (200, 31, 117)
    taps = synth.gaussian_taps(1.0)
    g = oracle_mod.texture_filter_rgb(rgb, 3, 5, 2, 1.0, 8.0, 5.0, 60.0, taps, lq_for(taps, 10.0), 10.0, 40.0)
    assert np.array_equal(g, rgb.astype(np.float64))


def test_texture_rgb_is_the_composition(oracle_mod):
    rgb = synth.make_rgb(14, 19, 21, n_blobs=5)
    taps = synth.gaussian_taps(1.0)
    Lq = lq_for(taps, 10.0)
    got = oracle_mod.texture_filter_rgb(rgb, 3, 4, 2, 1.0, 8.0, 5.0, 60.0, taps, Lq, 10.0, 40.0, sw=2, sN=5)
    s1 = oracle_mod.texture_sigma(oracle_mod.luma(rgb), 2, 1.0, 8.0, 5.0, 60.0)
    s2 = (s1 * np.float32(0.8)).astype(np.float32)
    f3 = np.empty_like(rgb)
    for c in range(3):
        f = np.ascontiguousarray(rgb[..., c])
        g1, _ = oracle_mod.fabf(f, f.astype(np.float32), s1, 3, 4)
        f2 = np.clip(np.rint(g1), 0, 255).astype(np.uint8)
        g2, _ = oracle_mod.fabf(f2, f2.astype(np.float32), s2, 3, 4)
        f3[..., c] = np.clip(np.rint(g2), 0, 255).astype(np.uint8)
    s3 = oracle_mod.sharpen_sigma(oracle_mod.luma(f3), taps, Lq, 10.0, 40.0)
    for c in range(3):
        f = np.ascontiguousarray(f3[..., c])
        ref, _ = oracle_mod.fabf(f, oracle_mod.sharpen_theta(f, 2), s3, 2, 5)
        assert np.array_equal(got[..., c], ref)


@pytest.mark.parametrize("H,W", [(1, 7), (6, 1)])
def test_texture_rgb_degenerate_shapes(oracle_mod, H, W):
    rgb = synth.make_rgb(H, W, 3, n_blobs=2)
    taps = synth.gaussian_taps(0.7)
    g = oracle_mod.texture_filter_rgb(rgb, 2, 3, 1, 1.0, 8.0, 5.0, 60.0, taps, lq_for(taps, 10.0), 10.0, 40.0)
    assert g.shape == (H, W, 3) and np.all(np.isfinite(g))
    assert g.min() >= -1e-9 and g.max() <= 255 + 1e-9
