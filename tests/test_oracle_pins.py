"""Pins of the CPU oracle against what the paper and mathematics fix
(no GPU).  Each test checks the oracle against something other than itself:
library routines (scipy's exact inverse Hilbert matrix, the truncated
normal distribution), exact rational arithmetic, brute force on tiny
inputs, mpmath quadrature, and closed-form limits."""
import json
import math
import os
from fractions import Fraction
from math import comb

import mpmath as mp
import numpy as np
import pytest
import scipy.linalg
import scipy.stats

from paper_1811_02308_gb300 import synth

U = 2.0 ** -53   # unit roundoff of binary64


def small_inputs(H, W, seed, sigma_range=(10.0, 40.0), zeta=None, n_blobs=4):
    return synth.make_inputs(H, W, seed, n_blobs=n_blobs, sigma_range=sigma_range, zeta_range=zeta)


def np_window(f, y, x, w):
    H, W = f.shape
    return f[max(0, y - w):min(H, y + w + 1), max(0, x - w):min(W, x + w + 1)].ravel()


# ---------------------------------------------------------------------------
# Hilbert inverse, Eqs. (18)-(19)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N", range(7))
def test_hilbert_inverse_equals_scipy_exact(oracle_mod, N):
    A = oracle_mod.hilbert_inverse(N)
    ref = scipy.linalg.invhilbert(N + 1, exact=True)
    assert [[int(v) for v in row] for row in A] == [[int(v) for v in row] for row in ref]


@pytest.mark.parametrize("N", range(7))
def test_hilbert_inverse_times_hilbert_is_identity(oracle_mod, N):
    A = oracle_mod.hilbert_inverse(N)
    n = N + 1
    for i in range(n):
        for j in range(n):
            s = sum(Fraction(int(A[i, k]), k + j + 1) for k in range(n))
            assert s == (1 if i == j else 0)


def test_hilbert_inverse_2x2(oracle_mod):
    assert oracle_mod.hilbert_inverse(1).tolist() == [[4, -6], [-6, 12]]


# ---------------------------------------------------------------------------
# Window statistics, Eqs. (8), (17), (24): brute force on tiny images
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("H,W,w,seed", [(7, 9, 1, 1), (7, 9, 3, 2), (1, 1, 2, 3), (1, 11, 2, 4),
                                        (12, 5, 4, 5), (13, 17, 6, 6), (5, 5, 40, 7)])
def test_window_statistics_bruteforce(oracle_mod, H, W, w, seed):
    f, _, _ = small_inputs(H, W, seed)
    N = 6
    a, b = oracle_mod.bounds(f, w)
    m = oracle_mod.moments(f, w, N)
    M = oracle_mod.shifted_moments(f, w, N)
    for y in range(H):
        for x in range(W):
            v = [int(t) for t in np_window(f, y, x, w)]
            assert a[y, x] == min(v) and b[y, x] == max(v)
            for k in range(N + 1):
                assert m[k, y, x] == sum(t ** k for t in v)
                assert M[k, y, x] == sum((t - min(v)) ** k for t in v)


def test_shifted_moments_binomial_form(oracle_mod):
    """Eq. (24) (Prop. in Sec. II-B): M_k = sum_r C(k,r) (-alpha)^(k-r) m_r."""
    f, _, _ = small_inputs(24, 31, 11)
    N, w = 6, 5
    a, _ = oracle_mod.bounds(f, w)
    m = oracle_mod.moments(f, w, N)
    M = oracle_mod.shifted_moments(f, w, N)
    for y in range(0, 24, 3):
        for x in range(0, 31, 2):
            al = int(a[y, x])
            for k in range(N + 1):
                ref = sum(comb(k, r) * (-al) ** (k - r) * int(m[r, y, x]) for r in range(k + 1))
                assert int(M[k, y, x]) == ref


def test_power_sums_exact_at_the_int64_limit(oracle_mod):
    """N = 6, w = 40 at the worst case (a window of 255s) fits int64 exactly."""
    f = np.full((81, 81), 255, np.uint8)
    f[0, 0] = 0
    m = oracle_mod.moments(f, 40, 6)
    assert int(m[6, 40, 40]) == 6560 * 255 ** 6
    M = oracle_mod.shifted_moments(f, 40, 6)
    assert int(M[6, 40, 40]) == 6560 * 255 ** 6


# ---------------------------------------------------------------------------
# Brute force, Eqs. (1)-(3): range-space form (Eqs. (5)-(7)) and rescaled
# form (Eqs. (20)-(27)) computed independently on tiny images
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("w", [1, 2, 4])
def test_bruteforce_equals_histogram_form(oracle_mod, w):
    f, th, s = small_inputs(9, 11, 21, zeta=(-20, 20))
    g = oracle_mod.bruteforce(f, th, s, w)
    for y in range(9):
        for x in range(11):
            v = np_window(f, y, x, w)
            h = np.bincount(v, minlength=256)          # Eq. (5), omega == 1
            t = np.nonzero(h)[0]
            theta, sig = mp.mpf(float(th[y, x])), mp.mpf(float(s[y, x]))
            num = mp.fsum(int(tt) * int(h[tt]) * mp.exp(-(tt - theta) ** 2 / (2 * sig * sig)) for tt in t)
            den = mp.fsum(int(h[tt]) * mp.exp(-(tt - theta) ** 2 / (2 * sig * sig)) for tt in t)
            ref = float(num / den)                     # Eqs. (6)-(7)
            assert abs(g[y, x] - ref) <= 1e-13 * abs(ref) + 1e-12
            # Eqs. (20)-(27): g = alpha + (beta - alpha) F on the stretched domain
            al, be = int(t.min()), int(t.max())
            if al == be:
                assert ref == pytest.approx(al, abs=1e-12)
                continue
            lam = mp.mpf((be - al) ** 2) / (2 * sig * sig)
            th0 = (theta - al) / (be - al)
            G = [(mp.mpf(int(tt) - al) / (be - al), int(h[tt])) for tt in t]
            F = mp.fsum(u * c * mp.exp(-lam * (u - th0) ** 2) for u, c in G) / \
                mp.fsum(c * mp.exp(-lam * (u - th0) ** 2) for u, c in G)
            assert abs(float(al + (be - al) * F) - ref) <= 1e-13 * abs(ref) + 1e-12


# ---------------------------------------------------------------------------
# Integrals, Eqs. (28), (30)-(32): against adaptive quadrature (mpmath)
# ---------------------------------------------------------------------------
def _quad_I(lam, t0, K):
    mp.mp.dps = 40
    lam, t0 = mp.mpf(lam), mp.mpf(t0)
    d = -t0 if t0 < 0 else (t0 - 1 if t0 > 1 else mp.mpf(0))
    pts = [0, 1]
    if 0 < t0 < 1:
        pts = [0, t0, 1]
    w = 1 / mp.sqrt(2 * lam)
    extra = [p for p in (t0 - 6 * w, t0 + 6 * w) if 0 < p < 1]
    pts = sorted(set(pts + extra))
    return [mp.quad(lambda t: t ** k * mp.exp(-lam * (t - t0) ** 2 + lam * d * d), pts)
            for k in range(K + 1)]


LAMS = [1e-7, 5e-5, 1.5e-4, 1e-3, 0.05, 0.5, 1.0, 5.0, 50.0, 1000.0]
T0S = [-3.0, -0.4, -0.05, 0.0, 0.3, 0.5, 1.0, 1.2, 5.0]


@pytest.mark.parametrize("lam", LAMS)
def test_integrals_match_quadrature(oracle_mod, lam):
    for t0 in T0S:
        d = -t0 if t0 < 0 else max(t0 - 1, 0.0)
        if lam * d * d > 50:      # oracle's stated domain: lambda d^2 <= 50
            continue
        got = oracle_mod.integrals(lam, t0, 7)
        ref = _quad_I(lam, t0, 7)
        for k in range(8):
            r = float(ref[k])
            assert abs(got[k] - r) <= 2e-15 * abs(r), (lam, t0, k, got[k], r)


def test_integrals_small_lambda_limit(oracle_mod):
    """lambda -> 0: I_k -> 1/(k+1) (the kernel becomes flat)."""
    got = oracle_mod.integrals(1e-14, 0.37, 7)
    for k in range(8):
        assert got[k] == pytest.approx(1.0 / (k + 1), rel=1e-12)


def test_integrals_satisfy_recursion_identity(oracle_mod):
    """Eq. (30) as an identity between the returned values, lambda = 3."""
    lam, t0 = 3.0, 0.41
    I = oracle_mod.integrals(lam, t0, 7)
    E1 = math.exp(-lam * (1 - t0) ** 2)
    for k in range(2, 8):
        rhs = t0 * I[k - 1] + (k - 1) / (2 * lam) * I[k - 2] - E1 / (2 * lam)
        assert I[k] == pytest.approx(rhs, rel=1e-13)


# ---------------------------------------------------------------------------
# Fit, Eqs. (14), (19), (24): moment matching
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_fit_matches_target_moments(oracle_mod, N):
    """c = A^{-1} mu (Eq. (19)) makes the moments of p equal mu (Eq. (14)).

    The exact solution c* = A^{-1} mu* is formed in rationals from scipy's
    exact inverse and the exact mu* = M_k / d^k; the oracle's FP64 c must lie
    within the rigorous forward-error bound of a fused dot product of N+1
    terms plus the rounding of mu, and the moments of the oracle's p must
    match mu* within the image of that bound."""
    f, th, s = small_inputs(32, 40, 31 + N, zeta=(-20, 20), sigma_range=(5, 60))
    rng = np.random.default_rng(N)
    Ainv = scipy.linalg.invhilbert(N + 1, exact=True)
    gamma = (N + 1) * U / (1 - (N + 1) * U)
    for _ in range(12):
        y, x = int(rng.integers(0, 32)), int(rng.integers(0, 40))
        tr = oracle_mod.fabf_trace(f, th, s, 5, N, y, x)
        if tr["flat"]:
            continue
        d = tr["beta"] - tr["alpha"]
        mu_ex = [Fraction(int(tr["M"][k]), d ** k) for k in range(N + 1)]
        for k in range(N + 1):
            assert abs(Fraction(tr["mu"][k]) - mu_ex[k]) <= 2 * U * mu_ex[k]
        bound = []
        for n in range(N + 1):
            c_ex = sum(Fraction(int(Ainv[n][k])) * mu_ex[k] for k in range(N + 1))
            scale = sum(abs(int(Ainv[n][k])) * mu_ex[k] for k in range(N + 1))
            b = (Fraction(gamma) + 2 * U * (1 + Fraction(gamma))) * scale
            assert abs(Fraction(tr["c"][n]) - c_ex) <= b, (n, float(tr["c"][n]), float(c_ex))
            bound.append(b)
        c = [Fraction(v) for v in tr["c"]]
        for k in range(N + 1):
            mom = sum(c[n] / (n + k + 1) for n in range(N + 1))
            assert abs(mom - mu_ex[k]) <= sum(bound[n] / (n + k + 1) for n in range(N + 1))
            # and the residual is far below the moment itself
            assert abs(mom - mu_ex[k]) <= Fraction(1, 10 ** 6) * mu_ex[0]


@pytest.mark.parametrize("N", [0, 1, 3, 6])
def test_fit_step_recovers_a_known_polynomial(oracle_mod, N):
    """The fit step alone: given the exact moments mu_k = int_0^1 t^k p(t) dt
    = sum_j c_j / (j + k + 1) of a polynomial p with small integer
    coefficients (rounded once to binary64), the oracle's fit returns those
    coefficients within the dot product's forward-error bound, and a common
    scale of the moments scales the coefficients (the fit is linear)."""
    rng = np.random.default_rng(90 + N)
    c_true = [int(v) for v in rng.integers(-9, 10, N + 1)]
    mu_ex = [sum(Fraction(c_true[j], j + k + 1) for j in range(N + 1)) for k in range(N + 1)]
    mu = np.array([float(v) for v in mu_ex])
    c = oracle_mod.fit(N, mu)
    Ainv = scipy.linalg.invhilbert(N + 1, exact=True)
    gamma = (N + 1) * U / (1 - (N + 1) * U)
    for n in range(N + 1):
        scale = sum(abs(int(Ainv[n][k])) * abs(mu_ex[k]) for k in range(N + 1))
        assert abs(Fraction(c[n]) - c_true[n]) <= (Fraction(gamma) + 2 * U * (1 + Fraction(gamma))) * scale
    c8 = oracle_mod.fit(N, mu * 8.0)       # a power-of-two scale is exact
    assert np.array_equal(c8, 8.0 * c)


# ---------------------------------------------------------------------------
# Whole Algorithm 1: special cases with closed forms
# ---------------------------------------------------------------------------
def test_constant_image_is_returned_unchanged(oracle_mod):
    f = np.full((20, 23), 137, np.uint8)
    th = f.astype(np.float32) + 3.0
    s = np.full(f.shape, 12.0, np.float32)
    g, nf = oracle_mod.fabf(f, th, s, 4, 5)
    assert nf == 0 and np.array_equal(g, f.astype(np.float64))


@pytest.mark.parametrize("N", [0, 1, 3, 5, 6])
def test_sigma_infinity_gives_box_mean(oracle_mod, N):
    """sigma -> inf: psi == 1, so by moment matching T1/T2 = mu_1/mu_0 and
    g_hat is the plain box mean m_1/m_0 (Eqs. (14), (29)) once N >= 1; for
    N = 0 only mu_0 is matched, p is constant and g_hat is the midrange."""
    f, th, _ = small_inputs(19, 26, 41)
    s = np.full(f.shape, 1e9, np.float32)
    g, _ = oracle_mod.fabf(f, th, s, 3, N)
    m = oracle_mod.moments(f, 3, 1)
    box = m[1] / m[0]
    a, b = oracle_mod.bounds(f, 3)
    flat = a == b
    ref = box if N >= 1 else (a.astype(np.float64) + b) / 2
    np.testing.assert_allclose(g[~flat], ref[~flat], rtol=1e-9)


def test_degree_zero_is_truncated_normal_mean(oracle_mod):
    """N = 0: p is constant, so T1/T2 = I_1/I_0 is the mean of a normal with
    mean t0 and variance 1/(2 lambda) truncated to [0, 1]."""
    f, th, s = small_inputs(21, 18, 51, zeta=(-10, 10))
    g, _ = oracle_mod.fabf(f, th, s, 2, 0)
    a, b = oracle_mod.bounds(f, 2)
    for y in range(21):
        for x in range(18):
            al, be = int(a[y, x]), int(b[y, x])
            if al == be:
                continue
            d = be - al
            t0 = (float(th[y, x]) - al) / d
            sd = math.sqrt(1.0 / (2.0 * (d * d / (2.0 * float(s[y, x]) ** 2))))
            mean = scipy.stats.truncnorm.mean((0 - t0) / sd, (1 - t0) / sd, loc=t0, scale=sd)
            assert g[y, x] == pytest.approx(al + d * mean, rel=1e-10, abs=1e-9)


def test_psnr_rises_with_degree_like_table1(oracle_mod):
    """Table I: PSNR(g_hat, g) grows with N.  Synthetic stand-in image,
    classical filter (theta = f), sigma = 40, box radius 5."""
    tab = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1_psnr.json")))
    assert all(np.diff(tab["rho=5"]) > 0)
    f, _, _ = small_inputs(96, 96, 61, n_blobs=8)
    th = f.astype(np.float32)
    s = np.full(f.shape, 40.0, np.float32)
    g = oracle_mod.bruteforce(f, th, s, 5)
    ps = []
    for N in range(7):
        gh, _ = oracle_mod.fabf(f, th, s, 5, N)
        ps.append(10 * math.log10(255.0 ** 2 / np.mean((gh - g) ** 2)))
    assert all(np.diff(ps) > 0), ps
    assert ps[5] >= 40.0, ps
