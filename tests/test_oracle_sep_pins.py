"""Pins of the oracle's separable-spatial-kernel functions (no GPU).

The spatial kernel omega(j) = g[jy + r] g[jx + r] with integer taps (Eq. (4)
when the taps are a quantised Gaussian).  Each test checks the oracle against
something other than itself: Python-integer brute force (exact, any size),
the box-kernel functions that tests/test_oracle_pins.py pins (all-ones taps),
closed-form limits (weighted mean, truncated normal), exact rationals for the
fit, numpy for the brute-force filter, and Table I's trend for the Gaussian.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

from paper_1811_02308_gb300 import synth


def small_inputs(H, W, seed, sigma_range=(10.0, 40.0), zeta=None, n_blobs=4):
    return synth.make_inputs(H, W, seed, n_blobs=n_blobs, sigma_range=sigma_range, zeta_range=zeta)


def window_weights(f, taps, y, x):
    """Window values and weights at (y, x), clipped to the image (Python ints)."""
    H, W = f.shape
    r = len(taps) // 2
    vals, wts = [], []
    for yy in range(max(0, y - r), min(H, y + r + 1)):
        for xx in range(max(0, x - r), min(W, x + r + 1)):
            vals.append(int(f[yy, xx]))
            wts.append(int(taps[yy - y + r]) * int(taps[xx - x + r]))
    return vals, wts


@pytest.mark.parametrize("H,W,r,seed", [(7, 9, 1, 1), (9, 8, 3, 2), (1, 1, 2, 3), (1, 11, 2, 4),
                                        (12, 5, 4, 5), (6, 7, 40, 7)])
def test_weighted_moments_python_ints(oracle_mod, H, W, r, seed):
    rng = np.random.default_rng(seed)
    f = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    taps = synth.random_taps(r, rng, hi=1600 // (2 * r + 1) + 3)
    N = 6
    m = oracle_mod.moments_sep(f, taps, N)
    for y in range(H):
        for x in range(W):
            vals, wts = window_weights(f, taps, y, x)
            for k in range(N + 1):
                assert m[k, y, x] == sum(wv * v ** k for v, wv in zip(vals, wts)), (y, x, k)


def test_weighted_moments_beyond_64_bits(oracle_mod):
    # the largest case allowed: taps summing to 65535, every pixel 255, N = 6:
    # m_6 = 65535^2 255^6 ~ 2^80 must be exact
    r = 40
    taps = np.full(2 * r + 1, 809, np.uint32)
    taps[r] = 65535 - 809 * 2 * r
    f = np.full((81, 81), 255, np.uint8)
    f[3, 5] = 0
    m = oracle_mod.moments_sep(f, taps, 6)
    vals, wts = window_weights(f, taps, 40, 40)
    for k in range(7):
        assert m[k, 40, 40] == sum(wv * v ** k for v, wv in zip(vals, wts))
    assert m[6, 40, 40] > 2 ** 79


def test_shifted_moments_and_mu_exact(oracle_mod):
    rng = np.random.default_rng(11)
    f, th, s = small_inputs(13, 15, 11, zeta=(-20, 20))
    taps = synth.random_taps(4, rng)
    for N in (1, 4, 6):
        for y, x in ((0, 0), (6, 7), (12, 14), (3, 11)):
            tr = oracle_mod.fabf_sep_trace(f, th, s, taps, N, y, x)
            vals, wts = window_weights(f, taps, y, x)
            al, be = min(vals), max(vals)
            assert (tr["alpha"], tr["beta"]) == (al, be)
            if al == be:
                continue
            d = be - al
            for k in range(N + 1):
                Mk = sum(wv * (v - al) ** k for v, wv in zip(vals, wts))
                assert tr["M"][k] == Mk
                # one rounding of M_k and of d^k, then one IEEE division
                assert tr["mu"][k] == float(Mk) / float(d ** k)


def test_all_ones_taps_equal_box_kernel(oracle_mod):
    f, th, s = small_inputs(20, 23, 21, zeta=(-20, 20), sigma_range=(5, 60))
    for w, N in ((1, 0), (3, 5), (6, 6)):
        taps = np.ones(2 * w + 1, np.uint32)
        g_sep, nf_sep = oracle_mod.fabf_sep(f, th, s, taps, N)
        g_box, nf_box = oracle_mod.fabf(f, th, s, w, N)
        assert np.array_equal(g_sep, g_box)
        assert nf_sep == nf_box
        assert np.array_equal(oracle_mod.bruteforce_sep(f, th, s, taps), oracle_mod.bruteforce(f, th, s, w))


@pytest.mark.parametrize("N", [2, 5, 6])
def test_weighted_fit_matches_exact_rationals(oracle_mod, N):
    # c = A^{-1} mu, Eq. (19): within the forward-error bound of an (N+1)-term
    # fused dot product of exact integers with correctly rounded mu
    f, th, s = small_inputs(15, 15, 31)
    taps = synth.gaussian_taps(1.5)
    Ainv = scipy.linalg.invhilbert(N + 1, exact=True)
    for y, x in ((7, 7), (0, 3), (14, 9)):
        tr = oracle_mod.fabf_sep_trace(f, th, s, taps, N, y, x)
        if tr["flat"]:
            continue
        mu = [Fraction(v) for v in tr["mu"]]
        for n in range(N + 1):
            exact = sum(Fraction(int(Ainv[n][k])) * mu[k] for k in range(N + 1))
            bound = (N + 1) * 2.0 ** -53 * sum(abs(int(Ainv[n][k])) * abs(float(mu[k])) for k in range(N + 1))
            assert abs(Fraction(tr["c"][n]) - exact) <= Fraction(bound) * (1 + Fraction(1, 1000))


def test_constant_image_is_returned(oracle_mod):
    f = np.full((11, 14), 201, np.uint8)
    th = f.astype(np.float32) - 7
    s = np.full(f.shape, 12.0, np.float32)
    g, nf = oracle_mod.fabf_sep(f, th, s, synth.gaussian_taps(2.0), 5)
    assert np.array_equal(g, f.astype(np.float64)) and nf == 0


@pytest.mark.parametrize("N", [1, 3, 6])
def test_sigma_infinity_gives_weighted_mean(oracle_mod, N):
    # As sigma -> infinity the range kernel is flat and Eq. (1) is the
    # omega-weighted mean; the fitted polynomial matches mu_0 and mu_1
    # exactly, so Algorithm 1 gives the same value.
    f, th, _ = small_inputs(12, 13, 41)
    s = np.full(f.shape, 1e9, np.float32)
    rng = np.random.default_rng(41)
    taps = synth.random_taps(3, rng)
    g, _ = oracle_mod.fabf_sep(f, th, s, taps, N)
    for y in range(12):
        for x in range(13):
            vals, wts = window_weights(f, taps, y, x)
            mean = Fraction(sum(wv * v for v, wv in zip(vals, wts)), sum(wts))
            assert g[y, x] == pytest.approx(float(mean), rel=1e-9)


def test_degree_zero_is_truncated_normal_mean(oracle_mod):
    # N = 0: p is the constant mu_0, so g is the mean of a normal(theta,
    # sigma) truncated to [alpha, beta] whatever the weights
    f, th, s = small_inputs(10, 12, 51, zeta=(-20, 20))
    taps = synth.gaussian_taps(1.0)
    g, _ = oracle_mod.fabf_sep(f, th, s, taps, 0)
    for y, x in ((1, 1), (4, 9), (9, 11)):
        vals, _ = window_weights(f, taps, y, x)
        al, be = min(vals), max(vals)
        if al == be:
            continue
        sd = float(s[y, x])
        t = float(th[y, x])
        ref = scipy.stats.truncnorm.mean((al - t) / sd, (be - t) / sd, loc=t, scale=sd)
        assert g[y, x] == pytest.approx(ref, rel=1e-10, abs=1e-9)


def test_weighted_bruteforce_numpy_and_histogram_form(oracle_mod):
    f, th, s = small_inputs(14, 16, 61, zeta=(-20, 20), sigma_range=(5, 60))
    rng = np.random.default_rng(61)
    taps = synth.random_taps(3, rng)
    g = oracle_mod.bruteforce_sep(f, th, s, taps)
    for y in range(14):
        for x in range(16):
            vals, wts = window_weights(f, taps, y, x)
            v = np.array(vals, np.float64)
            om = np.array(wts, np.float64)
            phi = np.exp(-(v - float(th[y, x])) ** 2 / (2 * float(s[y, x]) ** 2))
            assert g[y, x] == pytest.approx((om * phi * v).sum() / (om * phi).sum(), rel=1e-13)
            # range-space form: the omega-weighted histogram h(u), Sec. II
            h = np.zeros(256)
            np.add.at(h, np.array(vals), om)
            u = np.arange(256.0)
            pu = np.exp(-(u - float(th[y, x])) ** 2 / (2 * float(s[y, x]) ** 2))
            assert g[y, x] == pytest.approx((h * pu * u).sum() / (h * pu).sum(), rel=1e-12)
    gp = oracle_mod.bruteforce_sep_pixels(f, th, s, taps, [0, 13, 5], [0, 15, 9])
    assert np.array_equal(gp, np.array([g[0, 0], g[13, 15], g[5, 9]]))


def test_sep_pixels_equal_whole_image(oracle_mod):
    f, th, s = small_inputs(17, 19, 71, zeta=(-20, 20), sigma_range=(5, 60))
    taps = synth.gaussian_taps(2.0)
    g, nf = oracle_mod.fabf_sep(f, th, s, taps, 5)
    ys = np.repeat(np.arange(17), 19)
    xs = np.tile(np.arange(19), 17)
    gp, nfp = oracle_mod.fabf_sep_pixels(f, th, s, taps, 5, ys, xs)
    assert np.array_equal(gp, g.ravel()) and nfp == nf


@pytest.mark.parametrize("rho", [3, 5])
def test_gaussian_psnr_rises_with_degree_like_table1(oracle_mod, rho):
    """Table I (Gaussian spatial kernel rho, sigma = 40, theta = f): PSNR of
    Algorithm 1 against the brute-force filter grows with N and passes 40 dB
    by N = 3.  Synthetic stand-in image; only the trend is pinned."""
    tab = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1_psnr.json")))
    assert all(np.diff(tab["rho=%d" % rho]) > 0) and tab["rho=%d" % rho][3] > 40
    f, _, _ = small_inputs(72, 80, 62, n_blobs=8)
    th = f.astype(np.float32)
    s = np.full(f.shape, 40.0, np.float32)
    taps = synth.gaussian_taps(rho)
    g = oracle_mod.bruteforce_sep(f, th, s, taps)
    ps = []
    for N in range(7):
        gh, _ = oracle_mod.fabf_sep(f, th, s, taps, N)
        ps.append(10 * math.log10(255.0 ** 2 / np.mean((gh - g) ** 2)))
    assert all(np.diff(ps) > 0), ps
    assert ps[3] >= 40.0, ps


def test_gaussian_taps_shape():
    for rho in (0.4, 1.0, 2.5, 5.0, 40 / 3):
        g = synth.gaussian_taps(rho)
        r = math.ceil(3 * rho)
        assert len(g) == 2 * r + 1 and g[r] == 1024
        assert np.array_equal(g, g[::-1])
        assert all(np.diff(g[:r + 1].astype(np.int64)) >= 0)
        assert int(g.sum()) <= 65535
        # the taps follow Eq. (4) to within half a unit
        t = np.arange(-r, r + 1)
        assert np.max(np.abs(g - 1024 * np.exp(-t * t / (2 * rho * rho)))) <= 0.5


@pytest.mark.parametrize("taps", [np.ones(83, np.uint32), np.array([1, 0, 1], np.uint32),
                                  np.full(5, 20000, np.uint32), np.ones(4, np.uint32)])
def test_invalid_taps_rejected(oracle_mod, taps):
    f, th, s = small_inputs(5, 5, 1)
    with pytest.raises(ValueError):
        oracle_mod.fabf_sep(f, th, s, taps, 3)
