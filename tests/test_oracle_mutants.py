"""The oracle's pins catch plausible mistakes (no GPU).

Each case plants one mistake in a temporary copy of oracle/fabf_oracle.c
(a dropped factor, a flipped sign, an off-by-one index, a swapped operand,
a wrong bound), builds it, routes the oracle wrapper to that build and runs
a quick battery of the same checks as tests/test_oracle_pins.py.  Every
mutant must fail at least one check; the unmodified source must pass them
all.  The planted mistakes live only in this file and in temporary builds.
"""
import math
import os
import subprocess
import tempfile
from fractions import Fraction

import mpmath as mp
import numpy as np
import pytest
import scipy.linalg
import scipy.stats

import oracle
from paper_1811_02308_gb300 import synth

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "fabf_oracle.c")

MUTANTS = {
    "window end off by one": ("*y1 = y + w > H - 1 ? H - 1 : y + w;",
                              "*y1 = y + w > H - 1 ? H - 1 : y + w - 1;"),
    "min with the wrong comparison": ("if (v < a) a = v;", "if (v > a) a = v;"),
    "power index shifted": ("{ m[k] += p; p *= v; }", "{ p *= v; m[k] += p; }"),
    "shift by alpha - 1": ("- alpha, p = 1;", "- alpha + 1, p = 1;"),
    "Hilbert inverse sign": ("((m + n) % 2 == 0) ? 1 : -1", "((m + n) % 2 == 1) ? 1 : -1"),
    "Hilbert inverse binomials transposed": (
        "binom(N + m, N + 1 - n) * binom(N + n, N + 1 - m)",
        "binom(N + m, N + 1 - m) * binom(N + n, N + 1 - n)"),
    "Gauss-Legendre weight doubled": ("wt[i] = 1 / ((1 - x * x) * dp * dp);",
                                      "wt[i] = 2 / ((1 - x * x) * dp * dp);"),
    "erfc branch sign": ("diff = erfcf128(v) - erfcf128(u);", "diff = erfcf128(u) - erfcf128(v);"),
    "I_0 missing 1/2": ("I[0] = sqrtf128(pi / lam) / 2 * diff;", "I[0] = sqrtf128(pi / lam) * diff;"),
    "I_1 sign": ("(E0 - E1) / (2 * lam)", "(E1 - E0) / (2 * lam)"),
    "recursion index": ("((q128)(k - 1)) / (2 * lam)", "((q128)(k)) / (2 * lam)"),
    "recursion boundary sign": ("I[k - 2] - E1 / (2 * lam);", "I[k - 2] + E1 / (2 * lam);"),
    "E_1 square dropped": ("expf128(-lam * (1 - t0) * (1 - t0))", "expf128(-lam * (1 - t0))"),
    "scale sign": ("q128 s = expf128(lam * d * d);", "q128 s = expf128(-lam * d * d);"),
    "mu divisor": ("/* Eq. (24), R2 */\n        dk *= d;", "/* Eq. (24), R2 */\n        dk *= d + 1;"),
    "fit index": ("acc = fma((double)Ainv[n * (N + 1) + k], mu[k], acc);",
                  "acc = fma((double)Ainv[n * (N + 1) + k], mu[n], acc);"),
    "t0 from beta": ("- (double)alpha) / (double)d;", "- (double)(alpha + d)) / (double)d;"),
    "lambda without the 2": ("(double)(d * d) / (2.0 * s * s)", "(double)(d * d) / (s * s)"),
    "T1 index": ("T1 = fma(c[k - 1], I[k], T1);", "T1 = fma(c[k - 1], I[k - 1], T1);"),
    "ratio without alpha": ("*g_out = (double)alpha + (double)d * F;", "*g_out = (double)d * F;"),
    "fallback inverted": ("F = mu[1] / mu[0];", "F = mu[0] / mu[1];"),
    "brute force kernel width": ("                double phi = exp(-(v - th) * (v - th) / (2.0 * s * s))",
                                 "                double phi = exp(-(v - th) * (v - th) / (s * s))"),
    "brute force numerator": ("num += phi * v;", "num += phi * th;"),
    "flat branch skipped": ("if (alpha == beta) {\n        /* Sec. II-A and Algorithm 1",
                            "if (alpha == beta && alpha < 0) {\n        /* Sec. II-A and Algorithm 1"),
    "separable weight mirrored": (
        "om = (u128)taps[yy - y + r] * taps[xx - x + r];\n            u128 v = f[",
        "om = (u128)taps[y - yy + r] * taps[xx - x + r];\n            u128 v = f["),
    "separable shifted weight dropped": ("{ M[k] += om * p; p *= v; }", "{ M[k] += p; p *= v; }"),
    "separable moments truncated to 64 bits": (
        "mu[k] = (double)M[k] / (double)dk;          /* Eq. (24); M_k rounded once */",
        "mu[k] = (double)(uint64_t)M[k] / (double)dk;"),
    "separable brute force unweighted denominator": ("den += om * phi;", "den += phi;"),
    "separable tap sum limit": ("s > ORACLE_TAP_SUM_MAX", "s > 2 * ORACLE_TAP_SUM_MAX"),
    "sharpening centre sign": ("* m[0] - m[1];", "* m[0] + m[1];"),
    "LoG centre weight": ("S[1] + S[2] + S[3] + S[4] - 4 * S[0]", "S[1] + S[2] + S[3] + S[4] - 5 * S[0]"),
    "texture gradient direction": ("clampi(xx + 1, 0, W - 1)", "clampi(xx - 1, 0, W - 1)"),
    "LoG neighbour offset": ("const int dy[5] = {0, -1, 1, 0, 0}, dx[5] = {0, 0, 0, -1, 1};",
                             "const int dy[5] = {0, -1, 2, 0, 0}, dx[5] = {0, 0, 0, -1, 1};"),
    "sharpening saturation inverted": ("const int64_t q = L < Lq ? L : Lq;", "const int64_t q = L < Lq ? Lq : L;"),
    "sharpening centre factor": ("const int64_t num = 2 * (int64_t)f", "const int64_t num = 3 * (int64_t)f"),
    "mRTV with the gradient sum for its maximum": (
        "const float mrtv = (float)((int64_t)(fmax - fmin) * gmax)",
        "const float mrtv = (float)((int64_t)(fmax - fmin) * gsum)"),
    "mRTV epsilon dropped": ("((float)gsum + (float)eps);", "((float)gsum);"),
    "texture vertical gradient dropped": (
        "const int64_t g = (vx > v ? vx - v : v - vx) + (vy > v ? vy - v : v - vy);",
        "const int64_t g = (vx > v ? vx - v : v - vx);"),
    "texture width map reversed": ("u = 1.0f;\n            const float hi = (float)s_hi, lo = (float)s_lo;\n"
                                   "            sigma[(long)y * W + x] = hi - (hi - lo) * u;",
                                   "u = 1.0f;\n            const float hi = (float)s_hi, lo = (float)s_lo;\n"
                                   "            sigma[(long)y * W + x] = lo + (hi - lo) * u;"),
}

# ---------------------------------------------------------------------------
# quick battery (references computed once, independently of the oracle)
# ---------------------------------------------------------------------------
_REF = {}


def _refs():
    if _REF:
        return _REF
    mp.mp.dps = 40
    pts = [(3e-5, 0.4), (0.02, -2.0), (0.3, 0.6), (2.0, 1.3), (40.0, 0.2), (40.0, -0.3)]
    ints = {}
    for lam, t0 in pts:
        L, T = mp.mpf(lam), mp.mpf(t0)
        d = -T if T < 0 else (T - 1 if T > 1 else mp.mpf(0))
        ints[(lam, t0)] = [float(mp.quad(lambda t: t ** k * mp.exp(-L * (t - T) ** 2 + L * d * d),
                                         [0, min(max(T, 0), 1), 1])) for k in range(8)]
    _REF["ints"] = ints
    f, th, s = synth.make_inputs(11, 13, 5, n_blobs=3, zeta_range=(-20, 20), sigma_range=(5, 60))
    _REF["tiny"] = (f, th, s)
    return _REF


def _window(f, y, x, w):
    return f[max(0, y - w):y + w + 1, max(0, x - w):x + w + 1].astype(np.int64).ravel()


def map_properties():
    """Properties the Sec. IV maps' definitions fix whatever the evaluation
    order (the closed forms of tests/test_oracle_app_pins.py): the LoG of an
    affine image is 0 and of x^2 is 2 S^2 in the interior, theta = f on an
    affine image, sigma at its bounds for a zero and a saturated LoG, mRTV's
    closed forms on a ramp, a step and a stripe texture, and both width maps
    commute with transposition."""
    taps = synth.gaussian_taps(1.0)
    r = len(taps) // 2
    S = int(taps.sum())
    x = np.arange(16)
    plane = np.clip(np.add.outer(3 * np.arange(12), 7 * x), 0, 255).astype(np.uint8)
    para = np.tile((x * x).astype(np.uint8), (12, 1))
    inner = (slice(r + 1, 12 - r - 1), slice(r + 1, 16 - r - 1))
    assert np.all(oracle.sharpen_log(plane, taps)[inner] == 0)
    assert np.all(oracle.sharpen_log(para, taps)[inner] == 2 * S * S)
    assert np.all(oracle.sharpen_sigma(plane, taps, 1000, 10.0, 40.0)[inner] == np.float32(40.0))
    assert np.all(oracle.sharpen_sigma(para, taps, 2 * S * S, 10.0, 40.0)[inner] == np.float32(10.0))
    aff = np.add.outer(5 * np.arange(10), 9 * np.arange(14)).astype(np.uint8)
    assert np.array_equal(oracle.sharpen_theta(aff, 2)[2:8, 2:12], aff[2:8, 2:12].astype(np.float32))
    k, n, eps, msat, lo, hi = 1, 3, 1.0, 64.0, 5.0, 60.0
    Hh, Ww, b, h = 9, 18, 3, 90
    ramp = np.tile((b * np.arange(Ww)).astype(np.uint8), (Hh, 1))
    step = np.zeros((Hh, Ww), np.uint8)
    step[:, Ww // 2:] = h
    stripes = np.tile(((np.arange(Ww) % 2) * h).astype(np.uint8), (Hh, 1))
    for img, mr in ((ramp, 2 * k * b * b / (n * n * b + eps)), (step, h * h / (n * h + eps)),
                    (stripes, h * h / (n * n * h + eps))):
        sg = oracle.texture_sigma(img, k, eps, msat, lo, hi)[Hh // 2, Ww // 2]
        assert abs(float(sg) - (hi - (hi - lo) * min(mr / msat, 1.0))) <= 1e-5 * hi
    f = synth.make_inputs(15, 19, 8, n_blobs=4)[0]
    assert np.array_equal(oracle.texture_sigma(f.T.copy(), 2, 1.0, 8.0, 5.0, 60.0),
                          oracle.texture_sigma(f, 2, 1.0, 8.0, 5.0, 60.0).T)
    assert np.array_equal(oracle.sharpen_log(f.T.copy(), taps), oracle.sharpen_log(f, taps).T)


APPLICATION_MUTANTS = ["sharpening centre sign", "LoG centre weight", "texture gradient direction",
                       "texture width map reversed", "LoG neighbour offset", "sharpening saturation inverted",
                       "sharpening centre factor", "mRTV with the gradient sum for its maximum",
                       "mRTV epsilon dropped", "texture vertical gradient dropped"]


def battery():
    """Run every check; return the names of those that fail."""
    R = _refs()
    fails = []

    def check(name, fn):
        try:
            fn()
        except Exception:     # noqa: BLE001 - a broken build may raise anything
            fails.append(name)

    def hilbert():
        for N in range(7):
            ref = scipy.linalg.invhilbert(N + 1, exact=True)
            assert oracle.hilbert_inverse(N).tolist() == [[int(v) for v in r] for r in ref]

    def window_stats():
        f, _, _ = R["tiny"]
        a, b = oracle.bounds(f, 2)
        m = oracle.moments(f, 2, 6)
        M = oracle.shifted_moments(f, 2, 6)
        for y in range(f.shape[0]):
            for x in range(f.shape[1]):
                v = _window(f, y, x, 2)
                assert a[y, x] == v.min() and b[y, x] == v.max()
                for k in range(7):
                    assert m[k, y, x] == int((v ** k).sum())
                    assert M[k, y, x] == int(((v - v.min()) ** k).sum())

    def integrals():
        for (lam, t0), ref in R["ints"].items():
            got = oracle.integrals(lam, t0, 7)
            assert np.allclose(got, ref, rtol=1e-13, atol=0)

    def fit_moments():
        f, th, s = R["tiny"]
        for N in (2, 5):
            Ainv = scipy.linalg.invhilbert(N + 1, exact=True)
            for y, x in ((3, 4), (7, 9), (0, 0)):
                tr = oracle.fabf_trace(f, th, s, 3, N, y, x)
                if tr["flat"]:
                    continue
                d = tr["beta"] - tr["alpha"]
                v = _window(f, y, x, 3)
                assert tr["alpha"] == v.min() and tr["beta"] == v.max()
                mu = [Fraction(int(((v - v.min()) ** k).sum()), d ** k) for k in range(N + 1)]
                for n in range(N + 1):
                    c_ex = sum(Fraction(int(Ainv[n][k])) * mu[k] for k in range(N + 1))
                    scale = sum(abs(int(Ainv[n][k])) * mu[k] for k in range(N + 1))
                    assert abs(Fraction(tr["c"][n]) - c_ex) <= Fraction(2 ** -48) * scale
                assert tr["t0"] == pytest.approx((float(th[y, x]) - tr["alpha"]) / d, rel=1e-15)
                assert tr["lam"] == pytest.approx(d * d / (2.0 * float(s[y, x]) ** 2), rel=1e-15)

    def constant_image():
        f = np.full((9, 12), 77, np.uint8)
        g, _ = oracle.fabf(f, f.astype(np.float32) + 2, np.full(f.shape, 9.0, np.float32), 2, 4)
        assert np.array_equal(g, f.astype(np.float64))

    def box_mean_limit():
        f, th, _ = R["tiny"]
        s = np.full(f.shape, 1e9, np.float32)
        g, _ = oracle.fabf(f, th, s, 2, 3)
        for y in range(f.shape[0]):
            for x in range(f.shape[1]):
                v = _window(f, y, x, 2)
                if v.min() != v.max():
                    assert g[y, x] == pytest.approx(v.mean(), rel=1e-9)

    def truncated_normal():
        f, th, s = R["tiny"]
        g, _ = oracle.fabf(f, th, s, 2, 0)
        for y, x in ((2, 2), (5, 8), (10, 12)):
            v = _window(f, y, x, 2)
            al, d = int(v.min()), int(v.max() - v.min())
            if d == 0:
                continue
            t0 = (float(th[y, x]) - al) / d
            sd = float(s[y, x]) / d
            mean = scipy.stats.truncnorm.mean(-t0 / sd, (1 - t0) / sd, loc=t0, scale=sd)
            assert g[y, x] == pytest.approx(al + d * mean, rel=1e-10, abs=1e-9)

    def bruteforce():
        f, th, s = R["tiny"]
        g = oracle.bruteforce(f, th, s, 2)
        for y, x in ((1, 1), (6, 7), (10, 12)):
            v = _window(f, y, x, 2).astype(np.float64)
            wgt = np.exp(-(v - float(th[y, x])) ** 2 / (2 * float(s[y, x]) ** 2))
            assert g[y, x] == pytest.approx((wgt * v).sum() / wgt.sum(), rel=1e-13)

    def fallback_rule():
        # pixels whose T2 <= 0 return the box mean alpha + d mu_1/mu_0 (R5)
        f, th, s = synth.make_inputs(64, 80, 3, n_blobs=20, zeta_range=None, sigma_range=(10, 40))
        _, nf = oracle.fabf(f, th, s, 5, 5)
        assert nf > 0
        found = 0
        for y in range(64):
            for x in range(80):
                tr = oracle.fabf_trace(f, th, s, 5, 5, y, x)
                if tr["fallback"]:
                    v = _window(f, y, x, 5)
                    assert tr["g"] == pytest.approx(v.mean(), rel=1e-12)
                    found += 1
                    if found == 2:
                        return
        assert found > 0

    def separable():
        # weighted sums against Python integers (asymmetric taps), mu of a
        # 2^80-sized moment, the weighted brute force against numpy, the
        # weighted mean as sigma -> infinity, and the tap-sum limit
        f, th, s = R["tiny"]
        taps = np.array([3, 9, 1, 7, 2], np.uint32)
        m = oracle.moments_sep(f, taps, 6)
        g = oracle.bruteforce_sep(f, th, s, taps)
        gm, _ = oracle.fabf_sep(f, th, np.full(f.shape, 1e9, np.float32), taps, 3)
        for y, x in ((0, 0), (5, 6), (10, 12), (4, 1)):
            vals, wts = [], []
            for yy in range(max(0, y - 2), min(11, y + 3)):
                for xx in range(max(0, x - 2), min(13, x + 3)):
                    vals.append(int(f[yy, xx]))
                    wts.append(int(taps[yy - y + 2]) * int(taps[xx - x + 2]))
            for k in range(7):
                assert m[k, y, x] == sum(wv * v ** k for v, wv in zip(vals, wts))
            al = min(vals)
            tr = oracle.fabf_sep_trace(f, th, s, taps, 4, y, x)
            if not tr["flat"]:
                assert tr["M"][4] == sum(wv * (v - al) ** 4 for v, wv in zip(vals, wts))
            v = np.array(vals, float)
            om = np.array(wts, float)
            phi = np.exp(-(v - float(th[y, x])) ** 2 / (2 * float(s[y, x]) ** 2))
            assert g[y, x] == pytest.approx((om * phi * v).sum() / (om * phi).sum(), rel=1e-13)
            assert gm[y, x] == pytest.approx((om * v).sum() / om.sum(), rel=1e-9)
        wide = np.full((9, 9), 255, np.uint8)
        wide[0, 0] = 0
        big = np.full(9, 7000, np.uint32)
        tr = oracle.fabf_sep_trace(wide, wide.astype(np.float32), np.full((9, 9), 30.0, np.float32),
                                   big, 6, 4, 4)
        M6 = sum(int(big[yy]) * int(big[xx]) * int(wide[yy, xx]) ** 6 for yy in range(9) for xx in range(9))
        assert tr["mu"][6] == float(M6) / float(255 ** 6)
        try:
            oracle.fabf_sep(f, th, s, np.full(5, 20000, np.uint32), 3)
        except ValueError:
            pass
        else:
            raise AssertionError("taps summing to 100000 were accepted")

    def applications():
        # the Sec. IV maps against direct numpy evaluations of the same readings
        f, _, _ = R["tiny"]
        fi = f.astype(np.int64)
        H, W = f.shape
        th = oracle.sharpen_theta(f, 2)
        for y, x in ((0, 0), (5, 6), (10, 12)):
            win = fi[max(0, y - 2):y + 3, max(0, x - 2):x + 3]
            # binary32 holds both integers exactly; IEEE division rounds the quotient once
            num = 2 * int(fi[y, x]) * win.size - int(win.sum())
            assert th[y, x] == np.float32(num) / np.float32(win.size)
        taps = np.array([1, 4, 1], np.uint32)
        p = np.pad(fi, 1, mode="edge")
        S = sum(int(taps[a]) * int(taps[b]) * p[a:a + H, b:b + W] for a in range(3) for b in range(3))
        Sp = np.pad(S, 1, mode="edge")
        L = Sp[:-2, 1:-1] + Sp[2:, 1:-1] + Sp[1:-1, :-2] + Sp[1:-1, 2:] - 4 * S
        assert np.array_equal(oracle.sharpen_log(f, taps), L)
        gx = np.abs(np.concatenate([fi[:, 1:], fi[:, -1:]], axis=1) - fi)
        gy = np.abs(np.concatenate([fi[1:, :], fi[-1:, :]], axis=0) - fi)
        g = gx + gy
        ts = oracle.texture_sigma(f, 1, 1.0, 8.0, 5.0, 60.0)
        for y, x in ((0, 0), (5, 6), (10, 12), (3, 9)):
            sl = (slice(max(0, y - 1), y + 2), slice(max(0, x - 1), x + 2))
            f32 = np.float32
            mr = f32(int(fi[sl].max() - fi[sl].min()) * int(g[sl].max())) / (f32(int(g[sl].sum())) + f32(1.0))
            assert ts[y, x] == f32(60.0) - (f32(60.0) - f32(5.0)) * min(mr / f32(8.0), f32(1.0))

    for name, fn in [("map properties", map_properties),
                     ("hilbert", hilbert), ("window", window_stats), ("integrals", integrals),
                     ("fit", fit_moments), ("constant", constant_image), ("box mean", box_mean_limit),
                     ("truncated normal", truncated_normal), ("bruteforce", bruteforce),
                     ("fallback", fallback_rule), ("separable", separable), ("applications", applications)]:
        check(name, fn)
    return fails


def _build(src_text, tmpdir, tag):
    c = os.path.join(tmpdir, "m_%s.c" % tag)
    so = os.path.join(tmpdir, "m_%s.so" % tag)
    with open(c, "w") as fh:
        fh.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared", "-o", so, c,
                           "-lm"])
    return oracle.load_library(so)


@pytest.fixture(scope="module")
def source():
    oracle.build()
    return open(SRC).read()


def test_unmodified_oracle_passes_the_battery(source):
    with tempfile.TemporaryDirectory() as d:
        lib = _build(source, d, "orig")
        with oracle.use_library(lib):
            assert battery() == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(source, name):
    old, new = MUTANTS[name]
    assert source.count(old) == 1, "mutation site no longer unique: %r" % old
    with tempfile.TemporaryDirectory() as d:
        lib = _build(source.replace(old, new), d, "mut")
        with oracle.use_library(lib):
            fails = battery()
    assert fails, "planted mistake '%s' was not caught by any pin" % name


def test_unmodified_oracle_has_the_map_properties(source):
    with tempfile.TemporaryDirectory() as d:
        lib = _build(source, d, "orig_maps")
        with oracle.use_library(lib):
            map_properties()


@pytest.mark.parametrize("name", APPLICATION_MUTANTS)
def test_application_mutant_breaks_a_map_property(source, name):
    # the properties alone (no restatement of the maps' evaluation order)
    # catch each planted mistake in the Sec. IV maps
    old, new = MUTANTS[name]
    assert source.count(old) == 1, "mutation site no longer unique: %r" % old
    with tempfile.TemporaryDirectory() as d:
        lib = _build(source.replace(old, new), d, "mut_maps")
        with oracle.use_library(lib):
            with pytest.raises(Exception):
                map_properties()
