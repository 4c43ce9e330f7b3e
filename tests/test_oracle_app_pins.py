"""Pins of the oracle's application maps (Sec. IV; no GPU): the sharpening
centre and width (Sec. IV-A) and the texture width from mRTV (Sec. IV-C),
each against an independent numpy implementation of the same reading, bit
for bit, plus the behaviour the paper describes (flat regions get wide range
kernels, strong edges narrow ones; constant images pass unchanged)."""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1811_02308_gb300 import synth


def image(H, W, seed, n_blobs=4):
    f, _, _ = synth.make_inputs(H, W, seed, n_blobs=n_blobs)
    return f


def lq_for(taps, lap_sat):
    return int(math.floor(lap_sat * float(int(taps.sum())) ** 2 + 0.5))


def rn32(q: Fraction) -> np.float32:
    """The binary32 value nearest to the rational q (ties to even), found by
    exact comparison among the neighbours of a first guess."""
    c = np.float32(float(q))
    cands = [np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))]
    best = min(cands, key=lambda v: (abs(Fraction(float(v)) - q), int(np.frombuffer(v.tobytes(), np.uint32)[0]) & 1))
    return np.float32(best)


@pytest.mark.parametrize("H,W,w,seed", [(9, 11, 2, 1), (1, 7, 3, 2), (13, 5, 6, 3), (6, 6, 40, 4)])
def test_sharpen_theta_is_twice_f_minus_window_mean(oracle_mod, H, W, w, seed):
    f = image(H, W, seed)
    th = oracle_mod.sharpen_theta(f, w)
    for y in range(H):
        for x in range(W):
            win = f[max(0, y - w):y + w + 1, max(0, x - w):x + w + 1].astype(np.int64)
            m0, m1 = win.size, int(win.sum())
            ref = rn32(Fraction(2 * int(f[y, x]) * m0 - m1, m0))   # the exact quotient, rounded once
            assert th[y, x] == ref, (y, x)


def np_log(f, taps):
    """Integer Gaussian (clamped coordinates) then 5-point Laplacian (clamped)."""
    r = len(taps) // 2
    g = taps.astype(np.int64)
    H, W = f.shape
    p = np.pad(f.astype(np.int64), r, mode="edge")
    S = np.zeros((H, W), np.int64)
    for ty in range(2 * r + 1):
        for tx in range(2 * r + 1):
            S += g[ty] * g[tx] * p[ty:ty + H, tx:tx + W]
    Sp = np.pad(S, 1, mode="edge")
    return Sp[:-2, 1:-1] + Sp[2:, 1:-1] + Sp[1:-1, :-2] + Sp[1:-1, 2:] - 4 * S


@pytest.mark.parametrize("rho", [0.7, 1.0, 2.0])
def test_sharpen_log_and_sigma(oracle_mod, rho):
    f = image(17, 19, 5)
    taps = synth.gaussian_taps(rho)
    L = oracle_mod.sharpen_log(f, taps)
    assert np.array_equal(L, np_log(f, taps))
    Lq = lq_for(taps, 12.0)
    sg = oracle_mod.sharpen_sigma(f, taps, Lq, 10.0, 40.0)
    q = np.minimum(np.abs(L), Lq)
    f32 = np.float32
    u = q.astype(f32) / f32(Lq)                                  # binary32 operations, in order
    ref = f32(40.0) - (f32(40.0) - f32(10.0)) * u
    assert np.array_equal(sg, ref)
    assert sg.min() >= 10.0 and sg.max() <= 40.0


def np_texture_sigma(f, k, eps, msat, lo, hi):
    H, W = f.shape
    fi = f.astype(np.int64)
    gx = np.abs(np.concatenate([fi[:, 1:], fi[:, -1:]], axis=1) - fi)
    gy = np.abs(np.concatenate([fi[1:, :], fi[-1:, :]], axis=0) - fi)
    g = gx + gy
    out = np.zeros((H, W), np.float32)
    for y in range(H):
        for x in range(W):
            sl = (slice(max(0, y - k), y + k + 1), slice(max(0, x - k), x + k + 1))
            delta = int(fi[sl].max() - fi[sl].min())
            f32 = np.float32
            mrtv = f32(delta * int(g[sl].max())) / (f32(int(g[sl].sum())) + f32(eps))
            u = min(mrtv / f32(msat), f32(1.0))
            out[y, x] = f32(hi) - (f32(hi) - f32(lo)) * u
    return out


@pytest.mark.parametrize("k", [1, 2, 5])
def test_texture_sigma_from_mrtv(oracle_mod, k):
    f = image(15, 18, 7)
    got = oracle_mod.texture_sigma(f, k, 1.0, 8.0, 5.0, 60.0)
    assert np.array_equal(got, np_texture_sigma(f, k, 1.0, 8.0, 5.0, 60.0))


def test_maps_on_constant_and_step_images(oracle_mod):
    taps = synth.gaussian_taps(1.0)
    Lq = lq_for(taps, 10.0)
    c = np.full((12, 14), 90, np.uint8)
    assert np.array_equal(oracle_mod.sharpen_theta(c, 3), c.astype(np.float32))
    assert np.all(oracle_mod.sharpen_sigma(c, taps, Lq, 10.0, 40.0) == 40.0)      # flat: widest kernel
    assert np.all(oracle_mod.texture_sigma(c, 2, 1.0, 8.0, 5.0, 60.0) == 60.0)
    s = np.full((12, 14), 40, np.uint8)
    s[:, 7:] = 200                                                                 # a strong vertical edge
    sg = oracle_mod.sharpen_sigma(s, taps, Lq, 10.0, 40.0)
    assert sg[6, 6] == 10.0 and sg[6, 7] == 10.0 and sg[6, 0] == 40.0
    ts = oracle_mod.texture_sigma(s, 2, 1.0, 8.0, 5.0, 60.0)
    assert ts[6, 6] == 5.0 and ts[6, 0] == 60.0
    th = oracle_mod.sharpen_theta(s, 2)
    assert th[6, 6] < 40.0 and th[6, 7] > 200.0                                    # pushed apart


def test_texture_pipeline_keeps_constant_image(oracle_mod):
    c = np.full((10, 12), 137, np.uint8)
    taps = synth.gaussian_taps(1.0)
    g, mids = oracle_mod.texture_filter(c, 3, 5, 2, 1.0, 8.0, 5.0, 60.0, taps, lq_for(taps, 10.0), 10.0, 40.0)
    assert np.array_equal(g, c.astype(np.float64))
    assert all(np.array_equal(m, c.astype(np.float64)) for m in mids)


def test_texture_pipeline_is_the_composition(oracle_mod):
    f = image(16, 20, 9, n_blobs=6)
    taps = synth.gaussian_taps(1.0)
    Lq = lq_for(taps, 10.0)
    g, (g1, g2) = oracle_mod.texture_filter(f, 3, 4, 2, 1.0, 8.0, 5.0, 60.0, taps, Lq, 10.0, 40.0)
    s1 = oracle_mod.texture_sigma(f, 2, 1.0, 8.0, 5.0, 60.0)
    r1, _ = oracle_mod.fabf(f, f.astype(np.float32), s1, 3, 4)
    assert np.array_equal(r1, g1)
    f2 = np.clip(np.rint(r1), 0, 255).astype(np.uint8)
    r2, _ = oracle_mod.fabf(f2, f2.astype(np.float32), (s1 * np.float32(0.8)).astype(np.float32), 3, 4)
    assert np.array_equal(r2, g2)
    f3 = np.clip(np.rint(r2), 0, 255).astype(np.uint8)
    r3, _ = oracle_mod.fabf(f3, oracle_mod.sharpen_theta(f3, 3), oracle_mod.sharpen_sigma(f3, taps, Lq, 10.0, 40.0),
                            3, 4)
    assert np.array_equal(r3, g)


def test_texture_smoothing_removes_fine_texture(oracle_mod):
    # a flat region covered by fine texture (noise of std 10): mRTV is low
    # there, so the width map is wide and the two smoothing passes remove most
    # of the texture
    rng = np.random.default_rng(3)
    f = np.clip(np.rint(128 + rng.normal(0, 10, (24, 24))), 0, 255).astype(np.uint8)
    taps = synth.gaussian_taps(1.0)
    _, (g1, g2) = oracle_mod.texture_filter(f, 3, 5, 2, 1.0, 8.0, 5.0, 60.0, taps, lq_for(taps, 10.0), 10.0, 40.0)
    inner = (slice(4, 20), slice(4, 20))
    assert g2[inner].std() < 0.3 * f[inner].std()


# ---- properties the maps' definitions fix, independent of evaluation order

def test_log_of_planes_and_parabolas_in_the_interior(oracle_mod):
    # the Gaussian smoothing keeps an affine image affine (its taps are
    # symmetric) and the 5-point Laplacian of an affine function is 0; of x^2
    # it is 2 S^2 after smoothing with taps summing to S (second difference of
    # x^2 is 2, the tap sums multiply), away from the clamped borders
    taps = synth.gaussian_taps(1.0)
    r = len(taps) // 2
    S = int(taps.sum())
    x = np.arange(16)
    plane = np.clip(np.add.outer(3 * np.arange(12), 7 * x), 0, 255).astype(np.uint8)
    para = np.tile((x * x).astype(np.uint8), (12, 1))
    inner = (slice(r + 1, 12 - r - 1), slice(r + 1, 16 - r - 1))
    Lp = oracle_mod.sharpen_log(plane, taps)
    Lq = oracle_mod.sharpen_log(para, taps)
    assert np.all(Lp[inner] == 0)
    assert np.all(Lq[inner] == 2 * S * S)
    # a zero Laplacian gives the widest kernel, a saturated one the narrowest
    sg = oracle_mod.sharpen_sigma(plane, taps, lq_for(taps, 10.0), 10.0, 40.0)
    assert np.all(sg[inner] == np.float32(40.0))
    sq = oracle_mod.sharpen_sigma(para, taps, 2 * S * S, 10.0, 40.0)
    assert np.all(sq[inner] == np.float32(10.0))


def test_sharpen_theta_keeps_affine_images_in_the_interior(oracle_mod):
    # the window mean of an affine image over a symmetric window is its
    # centre value, so theta = 2 f - mean = f wherever the window is inside
    w = 2
    f = np.add.outer(5 * np.arange(10), 9 * np.arange(14)).astype(np.uint8)
    th = oracle_mod.sharpen_theta(f, w)
    inner = (slice(w, 10 - w), slice(w, 14 - w))
    assert np.array_equal(th[inner], f[inner].astype(np.float32))


def test_width_maps_are_monotone_and_bounded(oracle_mod):
    f = image(40, 50, 21, n_blobs=8)
    taps = synth.gaussian_taps(1.0)
    Lq = lq_for(taps, 4.0)
    L = np.abs(oracle_mod.sharpen_log(f, taps)).ravel()
    sg = oracle_mod.sharpen_sigma(f, taps, Lq, 10.0, 40.0).ravel()
    order = np.argsort(np.minimum(L, Lq), kind="stable")
    assert np.all(np.diff(sg[order].astype(np.float64)) <= 0)          # non-increasing in |LoG|
    assert sg.min() >= 10.0 and sg.max() <= 40.0
    ts = oracle_mod.texture_sigma(f, 2, 1.0, 8.0, 5.0, 60.0)
    assert ts.min() >= 5.0 and ts.max() <= 60.0


def test_maps_commute_with_transposition_and_offsets(oracle_mod):
    f = image(23, 31, 22, n_blobs=6)
    taps = synth.gaussian_taps(1.5)
    Lq = lq_for(taps, 6.0)
    assert np.array_equal(oracle_mod.sharpen_theta(f.T.copy(), 3), oracle_mod.sharpen_theta(f, 3).T)
    assert np.array_equal(oracle_mod.sharpen_log(f.T.copy(), taps), oracle_mod.sharpen_log(f, taps).T)
    assert np.array_equal(oracle_mod.texture_sigma(f.T.copy(), 2, 1.0, 8.0, 5.0, 60.0),
                          oracle_mod.texture_sigma(f, 2, 1.0, 8.0, 5.0, 60.0).T)
    # mirror images: the Laplacian of the symmetric smoothing is mirrored
    assert np.array_equal(oracle_mod.sharpen_log(f[:, ::-1].copy(), taps), oracle_mod.sharpen_log(f, taps)[:, ::-1])
    # an offset of the intensities moves theta by the offset and leaves the
    # widths unchanged (both depend on differences only)
    g = (f.astype(np.int64) // 2 + 20).astype(np.uint8)
    h = (g.astype(np.int64) + 37).astype(np.uint8)
    assert np.array_equal(oracle_mod.sharpen_sigma(h, taps, Lq, 10.0, 40.0),
                          oracle_mod.sharpen_sigma(g, taps, Lq, 10.0, 40.0))
    assert np.array_equal(oracle_mod.texture_sigma(h, 2, 1.0, 8.0, 5.0, 60.0),
                          oracle_mod.texture_sigma(g, 2, 1.0, 8.0, 5.0, 60.0))
    # (theta is one rounding of an exact quotient: the offset moves it within
    # two binary32 units of the values' binade)
    d = oracle_mod.sharpen_theta(h, 3).astype(np.float64) - oracle_mod.sharpen_theta(g, 3).astype(np.float64)
    assert np.all(np.abs(d - 37.0) <= 2 * float(np.spacing(np.float32(256))))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_mrtv_of_a_ramp_a_step_and_a_stripe_texture(oracle_mod, k):
    # closed forms of mRTV = delta * max|grad| / (sum|grad| + eps) over a
    # (2k+1)^2 window inside the image (forward differences):
    #   ramp f = b x:           delta = 2k b, max = b, sum = (2k+1)^2 b
    #   step of height h:       delta = h,    max = h, sum = (2k+1) h
    #   stripes 0, h, 0, h...:  delta = h,    max = h, sum = (2k+1)^2 h
    # and sigma = hi - (hi - lo) min(mRTV / msat, 1)
    n = 2 * k + 1
    eps, msat, lo, hi = 1.0, 64.0, 5.0, 60.0
    H, W = 4 * k + 5, 6 * k + 12
    b, h = 3, 90
    ramp = np.tile((b * np.arange(W)).astype(np.uint8), (H, 1))
    step = np.zeros((H, W), np.uint8)
    step[:, W // 2:] = h
    stripes = np.tile(((np.arange(W) % 2) * h).astype(np.uint8), (H, 1))
    y, xc = H // 2, W // 2
    cases = [(ramp, xc, 2 * k * b * b / (n * n * b + eps)),
             (step, xc, h * h / (n * h + eps)),
             (stripes, xc, h * h / (n * n * h + eps))]
    for img, x, mrtv in cases:
        sg = oracle_mod.texture_sigma(img, k, eps, msat, lo, hi)
        ref = hi - (hi - lo) * min(mrtv / msat, 1.0)
        assert abs(float(sg[y, x]) - ref) <= 1e-5 * hi, (k, mrtv, sg[y, x], ref)
    # an edge is far more structure than a fine texture of the same contrast
    s_step = oracle_mod.texture_sigma(step, k, eps, msat, lo, hi)[y, xc]
    s_tex = oracle_mod.texture_sigma(stripes, k, eps, msat, lo, hi)[y, xc]
    assert s_step < s_tex
