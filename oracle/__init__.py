"""ctypes wrapper of the plain CPU oracle (``fabf_oracle.c``).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA product
path (``paper_1811_02308_gb300``) never imports it.

All arrays are numpy; images are uint8 (H, W) with an optional row pitch,
``theta`` and ``sigma`` are float32 (H, W) C-contiguous.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fabf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

NMAX = 6
WMAX = 40


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source with gcc (no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


def load_library(path: str):
    """Load an oracle shared library and declare its signatures (the tests
    also load deliberately broken builds of the same source through this)."""
    lib = C.CDLL(path)
    u8p = C.POINTER(C.c_uint8)
    f32p = C.POINTER(C.c_float)
    f64p = C.POINTER(C.c_double)
    i64p = C.POINTER(C.c_int64)
    i32p = C.POINTER(C.c_int32)
    L = C.c_long
    I = C.c_int
    lib.oracle_hilbert_inverse.argtypes = [I, i64p]
    lib.oracle_integrals.argtypes = [C.c_double, C.c_double, I, f64p]
    lib.oracle_fit.argtypes = [I, f64p, f64p]
    lib.oracle_bounds.argtypes = [u8p, I, I, L, I, u8p, u8p]
    lib.oracle_moments.argtypes = [u8p, I, I, L, I, I, i64p]
    lib.oracle_shifted_moments.argtypes = [u8p, I, I, L, I, I, i64p]
    lib.oracle_fabf.argtypes = [u8p, f32p, f32p, I, I, L, I, I, f64p, C.POINTER(L)]
    lib.oracle_fabf_pixels.argtypes = [u8p, f32p, f32p, I, I, L, I, I, i32p, i32p, L,
                                       f64p, C.POINTER(L)]
    lib.oracle_fabf_trace.argtypes = [u8p, f32p, f32p, I, I, L, I, I, I, I, i32p, i64p,
                                      i64p, f64p, f64p, f64p, f64p, f64p, f64p, i32p]
    lib.oracle_bruteforce.argtypes = [u8p, f32p, f32p, I, I, L, I, f64p]
    lib.oracle_bruteforce_pixels.argtypes = [u8p, f32p, f32p, I, I, L, I, i32p, i32p, L,
                                             f64p]
    u32p = C.POINTER(C.c_uint32)
    u64p = C.POINTER(C.c_uint64)
    lib.oracle_moments_sep.argtypes = [u8p, I, I, L, u32p, I, I, u64p]
    lib.oracle_fabf_sep.argtypes = [u8p, f32p, f32p, I, I, L, u32p, I, I, f64p, C.POINTER(L)]
    lib.oracle_fabf_sep_pixels.argtypes = [u8p, f32p, f32p, I, I, L, u32p, I, I, i32p, i32p, L,
                                           f64p, C.POINTER(L)]
    lib.oracle_fabf_sep_trace.argtypes = [u8p, f32p, f32p, I, I, L, u32p, I, I, I, I, i32p, u64p,
                                          u64p, f64p, f64p, f64p, f64p, f64p, f64p, i32p]
    lib.oracle_bruteforce_sep.argtypes = [u8p, f32p, f32p, I, I, L, u32p, I, f64p]
    lib.oracle_bruteforce_sep_pixels.argtypes = [u8p, f32p, f32p, I, I, L, u32p, I, i32p, i32p,
                                                 L, f64p]
    lib.oracle_sharpen_theta.argtypes = [u8p, I, I, L, I, f32p]
    lib.oracle_sharpen_log.argtypes = [u8p, I, I, L, u32p, I, i64p]
    lib.oracle_sharpen_sigma.argtypes = [u8p, I, I, L, u32p, I, C.c_int64, C.c_double, C.c_double, f32p]
    lib.oracle_texture_sigma.argtypes = [u8p, I, I, L, I, C.c_double, C.c_double, C.c_double, C.c_double,
                                         f32p]
    for fn in (lib.oracle_sharpen_theta, lib.oracle_sharpen_log, lib.oracle_sharpen_sigma,
               lib.oracle_texture_sigma):
        fn.restype = C.c_int
    for fn in (lib.oracle_hilbert_inverse, lib.oracle_integrals, lib.oracle_bounds,
               lib.oracle_moments, lib.oracle_shifted_moments, lib.oracle_fabf,
               lib.oracle_fabf_pixels, lib.oracle_fabf_trace, lib.oracle_bruteforce,
               lib.oracle_bruteforce_pixels, lib.oracle_moments_sep, lib.oracle_fabf_sep,
               lib.oracle_fabf_sep_pixels, lib.oracle_fabf_sep_trace, lib.oracle_bruteforce_sep,
               lib.oracle_bruteforce_sep_pixels):
        fn.restype = C.c_int
    return lib


class use_library:
    """Context manager: route this module's functions to another build of the
    oracle (used only by the tests that plant mistakes)."""

    def __init__(self, lib):
        self.lib = lib

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = self.lib
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved


def _ptr(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def _maps(theta, sigma):
    return (np.ascontiguousarray(theta, dtype=np.float32),
            np.ascontiguousarray(sigma, dtype=np.float32))


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s rejected its arguments (rc=%d)" % (what, rc))


def hilbert_inverse(N: int) -> np.ndarray:
    """Closed-form inverse of the (N+1)x(N+1) Hilbert matrix, Eq. (19), int64."""
    out = np.zeros((N + 1, N + 1), dtype=np.int64)
    _check(_load().oracle_hilbert_inverse(N, _ptr(out, C.c_int64)), "hilbert_inverse")
    return out


def integrals(lam: float, t0: float, K: int) -> np.ndarray:
    """I_0..I_K of Eq. (28), each times exp(lambda d^2), d = dist(t0, [0,1])."""
    out = np.zeros(K + 1, dtype=np.float64)
    _check(_load().oracle_integrals(float(lam), float(t0), int(K), _ptr(out, C.c_double)),
           "integrals")
    return out


def fit(N: int, mu) -> np.ndarray:
    """The fit step of Algorithm 1 on given moments: c = A^{-1} mu (Eq. (19)),
    fused multiply-adds over ascending k; any common scale of mu carries
    through to c."""
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    c = np.zeros(N + 1, np.float64)
    _check(_load().oracle_fit(int(N), _ptr(mu, C.c_double), _ptr(c, C.c_double)), "fit")
    return c


def bounds(f, w):
    """alpha_i, beta_i of Eq. (8): window min and max, uint8 (H, W) each."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    a = np.zeros((H, W), np.uint8)
    b = np.zeros((H, W), np.uint8)
    _check(_load().oracle_bounds(_ptr(f, C.c_uint8), H, W, W, w, _ptr(a, C.c_uint8),
                                 _ptr(b, C.c_uint8)), "bounds")
    return a, b


def moments(f, w, N):
    """m_k of Eq. (17) (k = 0..N), int64 (N+1, H, W); m_0 is the window size."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    m = np.zeros((N + 1, H, W), np.int64)
    _check(_load().oracle_moments(_ptr(f, C.c_uint8), H, W, W, w, N, _ptr(m, C.c_int64)),
           "moments")
    return m


def shifted_moments(f, w, N):
    """M_k = sum over the window of (f - alpha)^k, int64 (N+1, H, W)."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    M = np.zeros((N + 1, H, W), np.int64)
    _check(_load().oracle_shifted_moments(_ptr(f, C.c_uint8), H, W, W, w, N,
                                          _ptr(M, C.c_int64)), "shifted_moments")
    return M


def fabf(f, theta, sigma, w, N):
    """Algorithm 1 on the whole image -> (g_hat float64 (H, W), n_fallback)."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    theta, sigma = _maps(theta, sigma)
    out = np.zeros((H, W), np.float64)
    nf = C.c_long(0)
    _check(_load().oracle_fabf(_ptr(f, C.c_uint8), _ptr(theta, C.c_float),
                               _ptr(sigma, C.c_float), H, W, W, w, N,
                               _ptr(out, C.c_double), C.byref(nf)), "fabf")
    return out, nf.value


def fabf_pixels(f, theta, sigma, w, N, ys, xs):
    """Algorithm 1 at pixels (ys[j], xs[j]) -> (values float64, n_fallback)."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    theta, sigma = _maps(theta, sigma)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    out = np.zeros(len(ys), np.float64)
    nf = C.c_long(0)
    _check(_load().oracle_fabf_pixels(_ptr(f, C.c_uint8), _ptr(theta, C.c_float),
                                      _ptr(sigma, C.c_float), H, W, W, w, N,
                                      _ptr(ys, C.c_int32), _ptr(xs, C.c_int32), len(ys),
                                      _ptr(out, C.c_double), C.byref(nf)), "fabf_pixels")
    return out, nf.value


def fabf_trace(f, theta, sigma, w, N, y, x):
    """Every intermediate of Algorithm 1 at one pixel, as a dict."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    theta, sigma = _maps(theta, sigma)
    ab = np.zeros(2, np.int32)
    m = np.zeros(N + 1, np.int64)
    M = np.zeros(N + 1, np.int64)
    mu = np.full(N + 1, np.nan)
    c = np.full(N + 1, np.nan)
    t0lam = np.full(2, np.nan)
    I = np.full(N + 2, np.nan)
    T = np.full(2, np.nan)
    g = np.zeros(1)
    fl = np.zeros(1, np.int32)
    _check(_load().oracle_fabf_trace(
        _ptr(f, C.c_uint8), _ptr(theta, C.c_float), _ptr(sigma, C.c_float), H, W, W, w, N,
        int(y), int(x), _ptr(ab, C.c_int32), _ptr(m, C.c_int64), _ptr(M, C.c_int64),
        _ptr(mu, C.c_double), _ptr(c, C.c_double), _ptr(t0lam, C.c_double),
        _ptr(I, C.c_double), _ptr(T, C.c_double), _ptr(g, C.c_double),
        _ptr(fl, C.c_int32)), "fabf_trace")
    return dict(alpha=int(ab[0]), beta=int(ab[1]), m=m, M=M, mu=mu, c=c, t0=t0lam[0],
                lam=t0lam[1], I=I, T1=T[0], T2=T[1], g=g[0], flat=bool(fl[0] & 1),
                fallback=bool(fl[0] & 2))


def bruteforce(f, theta, sigma, w):
    """Brute-force adaptive bilateral filter, Eqs. (1)-(3), float64 (H, W)."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    theta, sigma = _maps(theta, sigma)
    out = np.zeros((H, W), np.float64)
    _check(_load().oracle_bruteforce(_ptr(f, C.c_uint8), _ptr(theta, C.c_float),
                                     _ptr(sigma, C.c_float), H, W, W, w,
                                     _ptr(out, C.c_double)), "bruteforce")
    return out


def bruteforce_pixels(f, theta, sigma, w, ys, xs):
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    theta, sigma = _maps(theta, sigma)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    out = np.zeros(len(ys), np.float64)
    _check(_load().oracle_bruteforce_pixels(_ptr(f, C.c_uint8), _ptr(theta, C.c_float),
                                            _ptr(sigma, C.c_float), H, W, W, w,
                                            _ptr(ys, C.c_int32), _ptr(xs, C.c_int32),
                                            len(ys), _ptr(out, C.c_double)),
           "bruteforce_pixels")
    return out


def fabf_passes(f, theta, sigma, w, N, passes, sigma_decay=0.8):
    """Iterated filtering (texture filtering, Sec. IV-C): pass p+1 filters the
    previous output rounded half to even and clamped to [0, 255], with centre
    f_{p+1} + (theta - f) and width sigma_p * sigma_decay.  Returns the last
    pass's output (float64)."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    zeta = np.asarray(theta, np.float32) - f.astype(np.float32)
    th = np.asarray(theta, np.float32)
    sg = np.asarray(sigma, np.float32)
    g = None
    for p in range(passes):
        if p > 0:
            f = np.clip(np.rint(g), 0, 255).astype(np.uint8)
            th = (f.astype(np.float32) + zeta).astype(np.float32)
            sg = (sg * np.float32(sigma_decay)).astype(np.float32)
        g, _ = fabf(f, th, sg, w, N)
    return g


# ---------------------------------------------------------------------------
# Separable spatial kernel omega(j) = g[jy + r] g[jx + r] on [-r, r]^2
# (Eq. (4) for quantised Gaussian taps); taps are 2r+1 integers >= 0 with
# g[r] >= 1 and sum <= 65535.
# ---------------------------------------------------------------------------
def _taps(taps):
    t = np.ascontiguousarray(taps, dtype=np.uint32)
    if t.ndim != 1 or len(t) % 2 != 1:
        raise ValueError("taps must be a 1-D array of odd length 2r+1")
    return t, len(t) // 2


def _u128(words):
    """(..., 2) uint64 (low, high) -> Python ints (object array)."""
    lo = words[..., 0].astype(object)
    hi = words[..., 1].astype(object)
    return lo + (hi << 64)


def moments_sep(f, taps, N):
    """m_k = sum omega(j) f(i+j)^k (k = 0..N) as Python ints, object (N+1, H, W)."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    t, r = _taps(taps)
    m = np.zeros((N + 1, H, W, 2), np.uint64)
    _check(_load().oracle_moments_sep(_ptr(f, C.c_uint8), H, W, W, _ptr(t, C.c_uint32), r, N,
                                      _ptr(m, C.c_uint64)), "moments_sep")
    return _u128(m)


def fabf_sep(f, theta, sigma, taps, N):
    """Algorithm 1 with the separable kernel -> (g_hat float64 (H, W), n_fallback)."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    theta, sigma = _maps(theta, sigma)
    t, r = _taps(taps)
    out = np.zeros((H, W), np.float64)
    nf = C.c_long(0)
    _check(_load().oracle_fabf_sep(_ptr(f, C.c_uint8), _ptr(theta, C.c_float),
                                   _ptr(sigma, C.c_float), H, W, W, _ptr(t, C.c_uint32), r, N,
                                   _ptr(out, C.c_double), C.byref(nf)), "fabf_sep")
    return out, nf.value


def fabf_sep_pixels(f, theta, sigma, taps, N, ys, xs):
    """Algorithm 1 with the separable kernel at pixels (ys[j], xs[j])."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    theta, sigma = _maps(theta, sigma)
    t, r = _taps(taps)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    out = np.zeros(len(ys), np.float64)
    nf = C.c_long(0)
    _check(_load().oracle_fabf_sep_pixels(_ptr(f, C.c_uint8), _ptr(theta, C.c_float),
                                          _ptr(sigma, C.c_float), H, W, W, _ptr(t, C.c_uint32),
                                          r, N, _ptr(ys, C.c_int32), _ptr(xs, C.c_int32),
                                          len(ys), _ptr(out, C.c_double), C.byref(nf)),
           "fabf_sep_pixels")
    return out, nf.value


def fabf_sep_trace(f, theta, sigma, taps, N, y, x):
    """Every intermediate with the separable kernel at one pixel (m, M as ints)."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    theta, sigma = _maps(theta, sigma)
    t, r = _taps(taps)
    ab = np.zeros(2, np.int32)
    m = np.zeros((N + 1, 2), np.uint64)
    M = np.zeros((N + 1, 2), np.uint64)
    mu = np.full(N + 1, np.nan)
    c = np.full(N + 1, np.nan)
    t0lam = np.full(2, np.nan)
    I = np.full(N + 2, np.nan)
    T = np.full(2, np.nan)
    g = np.zeros(1)
    fl = np.zeros(1, np.int32)
    _check(_load().oracle_fabf_sep_trace(
        _ptr(f, C.c_uint8), _ptr(theta, C.c_float), _ptr(sigma, C.c_float), H, W, W,
        _ptr(t, C.c_uint32), r, N, int(y), int(x), _ptr(ab, C.c_int32), _ptr(m, C.c_uint64),
        _ptr(M, C.c_uint64), _ptr(mu, C.c_double), _ptr(c, C.c_double),
        _ptr(t0lam, C.c_double), _ptr(I, C.c_double), _ptr(T, C.c_double),
        _ptr(g, C.c_double), _ptr(fl, C.c_int32)), "fabf_sep_trace")
    flat = bool(fl[0] & 1)
    return dict(alpha=int(ab[0]), beta=int(ab[1]), m=list(_u128(m)),
                M=None if flat else list(_u128(M)), mu=mu, c=c, t0=t0lam[0], lam=t0lam[1],
                I=I, T1=T[0], T2=T[1], g=g[0], flat=flat, fallback=bool(fl[0] & 2))


def bruteforce_sep(f, theta, sigma, taps):
    """Brute-force filter, Eqs. (1)-(3), with the separable kernel, float64 (H, W)."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    theta, sigma = _maps(theta, sigma)
    t, r = _taps(taps)
    out = np.zeros((H, W), np.float64)
    _check(_load().oracle_bruteforce_sep(_ptr(f, C.c_uint8), _ptr(theta, C.c_float),
                                         _ptr(sigma, C.c_float), H, W, W, _ptr(t, C.c_uint32),
                                         r, _ptr(out, C.c_double)), "bruteforce_sep")
    return out


def bruteforce_sep_pixels(f, theta, sigma, taps, ys, xs):
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    theta, sigma = _maps(theta, sigma)
    t, r = _taps(taps)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    out = np.zeros(len(ys), np.float64)
    _check(_load().oracle_bruteforce_sep_pixels(_ptr(f, C.c_uint8), _ptr(theta, C.c_float),
                                                _ptr(sigma, C.c_float), H, W, W,
                                                _ptr(t, C.c_uint32), r, _ptr(ys, C.c_int32),
                                                _ptr(xs, C.c_int32), len(ys),
                                                _ptr(out, C.c_double)), "bruteforce_sep_pixels")
    return out


# ---------------------------------------------------------------------------
# Applications (Sec. IV): centre and width maps, sharpening, texture filtering
# ---------------------------------------------------------------------------
def sharpen_theta(f, w):
    """Sec. IV-A: theta = f + (f - mean of f over the clipped window), float32."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    out = np.zeros((H, W), np.float32)
    _check(_load().oracle_sharpen_theta(_ptr(f, C.c_uint8), H, W, W, w, _ptr(out, C.c_float)),
           "sharpen_theta")
    return out


def sharpen_log(f, taps):
    """Integer Laplacian of the integer-Gaussian-smoothed image (int64)."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    t, r = _taps(taps)
    out = np.zeros((H, W), np.int64)
    _check(_load().oracle_sharpen_log(_ptr(f, C.c_uint8), H, W, W, _ptr(t, C.c_uint32), r,
                                      _ptr(out, C.c_int64)), "sharpen_log")
    return out


def sharpen_sigma(f, taps, Lq, s_lo, s_hi):
    """Sec. IV-A: sigma = s_hi - (s_hi - s_lo) min(|LoG|, Lq) / Lq, float32."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    t, r = _taps(taps)
    out = np.zeros((H, W), np.float32)
    _check(_load().oracle_sharpen_sigma(_ptr(f, C.c_uint8), H, W, W, _ptr(t, C.c_uint32), r, int(Lq),
                                        float(s_lo), float(s_hi), _ptr(out, C.c_float)), "sharpen_sigma")
    return out


def texture_sigma(f, k, eps, msat, s_lo, s_hi):
    """Sec. IV-C: sigma from mRTV over the clipped window [-k, k]^2, float32."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    H, W = f.shape
    out = np.zeros((H, W), np.float32)
    _check(_load().oracle_texture_sigma(_ptr(f, C.c_uint8), H, W, W, int(k), float(eps), float(msat),
                                        float(s_lo), float(s_hi), _ptr(out, C.c_float)), "texture_sigma")
    return out


def _next_input(g):
    """Pass p+1 input: the output rounded half to even, clamped to [0, 255] (R9)."""
    return np.clip(np.rint(g), 0, 255).astype(np.uint8)


def sharpen(f, w, N, taps, Lq, s_lo, s_hi):
    """One sharpening pass (Sec. IV-A): Algorithm 1 with the maps above."""
    th = sharpen_theta(f, w)
    sg = sharpen_sigma(f, taps, Lq, s_lo, s_hi)
    g, _ = fabf(f, th, sg, w, N)
    return g


def texture_filter(f, w, N, k, eps, msat, t_lo, t_hi, taps, Lq, s_lo, s_hi, sigma_decay=0.8):
    """Texture filtering (Sec. IV-C): two smoothing passes with theta = f and
    the mRTV width map (scaled by sigma_decay on the second pass), then one
    sharpening pass.  Returns (g_final, [intermediate outputs])."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    s1 = texture_sigma(f, k, eps, msat, t_lo, t_hi)
    g1, _ = fabf(f, f.astype(np.float32), s1, w, N)
    f2 = _next_input(g1)
    s2 = (s1 * np.float32(sigma_decay)).astype(np.float32)
    g2, _ = fabf(f2, f2.astype(np.float32), s2, w, N)
    f3 = _next_input(g2)
    g3 = sharpen(f3, w, N, taps, Lq, s_lo, s_hi)
    return g3, [g1, g2]


# ---------------------------------------------------------------------------
# Colour (Sec. IV-C): channel by channel, width maps on the gray version
# ---------------------------------------------------------------------------
def luma(rgb):
    """Gray version of an interleaved 8-bit colour image (H, W, 3): the
    BT.601 luma 0.299 R + 0.587 G + 0.114 B rounded half up, computed in
    integers as floor((299 R + 587 G + 114 B + 500) / 1000)."""
    x = np.asarray(rgb).astype(np.int64)
    return ((299 * x[..., 0] + 587 * x[..., 1] + 114 * x[..., 2] + 500) // 1000).astype(np.uint8)


def _channel(rgb, c):
    return np.ascontiguousarray(np.asarray(rgb)[..., c], dtype=np.uint8)


def filter_rgb(rgb, theta, sigma, w, N):
    """Algorithm 1 on each channel of a colour image (Sec. IV-C).  theta is
    float32 (H, W, 3), or None for theta_c = f_c; sigma is one float32 (H, W)
    map shared by the channels.  Returns float64 (H, W, 3)."""
    H, W, _ = np.asarray(rgb).shape
    out = np.empty((H, W, 3), np.float64)
    for c in range(3):
        f = _channel(rgb, c)
        th = f.astype(np.float32) if theta is None else np.ascontiguousarray(np.asarray(theta)[..., c], np.float32)
        out[..., c], _ = fabf(f, th, sigma, w, N)
    return out


def texture_filter_rgb(rgb, w, N, k, eps, msat, t_lo, t_hi, taps, Lq, s_lo, s_hi, sigma_decay=0.8,
                       sw=None, sN=None):
    """Texture filtering of a colour image (Sec. IV-C): the mRTV width map
    of the luma; per channel the two smoothing passes (theta = f_c); the
    sharpening width map of the luma of the rounded second outputs, shared by
    the channels, with each channel's own sharpening centre.  sw, sN: the
    sharpening pass's radius and degree (default w, N).  Returns float64
    (H, W, 3)."""
    sw = w if sw is None else sw
    sN = N if sN is None else sN
    H, W, _ = np.asarray(rgb).shape
    s1 = texture_sigma(luma(rgb), k, eps, msat, t_lo, t_hi)
    s2 = (s1 * np.float32(sigma_decay)).astype(np.float32)
    f3 = np.empty((H, W, 3), np.uint8)
    for c in range(3):
        f = _channel(rgb, c)
        g1, _ = fabf(f, f.astype(np.float32), s1, w, N)
        f2 = _next_input(g1)
        g2, _ = fabf(f2, f2.astype(np.float32), s2, w, N)
        f3[..., c] = _next_input(g2)
    s3 = sharpen_sigma(luma(f3), taps, Lq, s_lo, s_hi)
    out = np.empty((H, W, 3), np.float64)
    for c in range(3):
        f = _channel(f3, c)
        out[..., c], _ = fabf(f, sharpen_theta(f, sw), s3, sw, sN)
    return out
