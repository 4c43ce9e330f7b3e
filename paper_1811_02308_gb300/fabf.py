"""Thin Python binding of ``libfabf.so`` (include/fabf.h): ctypes argument
marshalling only.  Every step of the filter runs in the CUDA kernels; if the
library is missing or cannot be loaded this module raises -- there is no CPU
fallback.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; CUDA tensors are
passed to the library as device pointers, everything else as host pointers.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

FABF_OK = 0
FABF_EINVAL = 1
FABF_ENOMEM = 2
FABF_EAGAIN = 3
FABF_EUNSUPPORTED = 4
FABF_ECUDA = 5
FABF_ETIMEOUT = 6
FABF_ENOTFOUND = 7

FABF_FP64 = 0
FABF_FP64FIT_FP32REC = 1
FABF_CFP32 = 2
FABF_C32 = 3

_lib = None


class FabfError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__("%s failed: %s (status %d)" % (what, status_str(status), status))


class _Config(C.Structure):
    _fields_ = [("device", C.c_int), ("mem_budget_bytes", C.c_size_t), ("precision", C.c_int),
                ("autotune", C.c_int), ("tune_cache_path", C.c_char_p)]


class Request(C.Structure):
    """``fabf_request`` of include/fabf.h."""
    _fields_ = [("img", C.c_void_p), ("theta", C.c_void_p), ("sigma", C.c_void_p),
                ("H", C.c_int), ("W", C.c_int), ("pitch", C.c_size_t), ("w", C.c_int),
                ("N", C.c_int), ("passes", C.c_int), ("sigma_decay", C.c_float),
                ("out", C.c_void_p), ("out_is_f64", C.c_int)]


class SharpenCfg(C.Structure):
    """fabf_sharpen_cfg (Sec. IV-A sharpening maps)."""
    _fields_ = [("w", C.c_int), ("N", C.c_int), ("rho_log", C.c_double), ("lap_sat", C.c_double),
                ("sigma_lo", C.c_double), ("sigma_hi", C.c_double)]


class TextureCfg(C.Structure):
    """fabf_texture_cfg (Sec. IV-C texture filtering)."""
    _fields_ = [("w", C.c_int), ("N", C.c_int), ("k", C.c_int), ("eps", C.c_double), ("mrtv_sat", C.c_double),
                ("sigma_lo", C.c_double), ("sigma_hi", C.c_double), ("sigma_decay", C.c_double),
                ("sharpen", SharpenCfg)]


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libfabf.so (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libfabf.so not found at %s: run paper_1811_02308_gb300.build.build() "
                           "(the CUDA library is required; there is no CPU fallback)" % path)
    lib = C.CDLL(path)
    vp, i, sz = C.c_void_p, C.c_int, C.c_size_t
    sig = {
        "fabf_create": ([C.POINTER(_Config), C.POINTER(vp)], i),
        "fabf_destroy": ([vp], i),
        "fabf_set_precision": ([vp, i], i),
        "fabf_filter": ([vp, vp, vp, vp, i, i, sz, i, i, vp, i, vp], i),
        "fabf_get_status": ([vp, vp, C.POINTER(i), C.POINTER(C.c_uint64)], i),
        "fabf_get_status_ex": ([vp, vp, C.POINTER(i), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)], i),
        "fabf_filter_batch": ([vp, C.POINTER(Request), i, vp], i),
        "fabf_serve_submit": ([vp, C.POINTER(Request), C.POINTER(C.c_uint64)], i),
        "fabf_serve_poll": ([vp, C.c_uint64, i, C.POINTER(i)], i),
        "fabf_status_str": ([i], C.c_char_p),
        "fabf_filter_noalloc": ([vp, vp, vp, i, i, sz, i, i, vp, i, vp, C.POINTER(C.c_uint64)], i),
        "fabf_serve_stats": ([vp, C.POINTER(C.c_uint64), C.POINTER(i)], i),
        "fabf_batch_stats": ([vp, C.POINTER(i), C.POINTER(i)], i),
        "fabf_tile_rows": ([vp, i, i, i, C.POINTER(i)], i),
        "fabf_hilbert_inverse": ([i, vp], i),
        "fabf_centred_inverse": ([i, vp], i),
        "fabf_fused_smem_bytes": ([i, i, C.POINTER(sz)], i),
        "fabf_debug_stages": ([vp, vp, vp, vp, i, i, sz, i, i] + [vp] * 11, i),
        "fabf_debug_integrals": ([vp, vp, vp, C.c_int64, i, i, vp], i),
        "fabf_bruteforce": ([vp, vp, vp, vp, i, i, sz, i, vp, i, i, vp], i),
        "fabf_filter_sep": ([vp, vp, vp, vp, i, i, sz, vp, i, i, vp, i, vp], i),
        "fabf_gaussian_taps": ([C.c_double, vp, i, C.POINTER(i)], i),
        "fabf_debug_stages_sep": ([vp, vp, vp, vp, i, i, sz, vp, i, i] + [vp] * 11, i),
        "fabf_bruteforce_sep": ([vp, vp, vp, vp, i, i, sz, vp, i, vp, i, i, vp], i),
        "fabf_filter_cascade": ([vp, vp, vp, vp, i, i, sz, i, i, vp, i, i, vp], i),
        "fabf_debug_fp64_functions": ([vp, vp, C.c_int64, vp, vp], i),
        "fabf_cascade_taps": ([i, vp, i, C.POINTER(i)], i),
        "fabf_cascade_radius": ([C.c_double, C.POINTER(i)], i),
        "fabf_debug_stages_cascade": ([vp, vp, vp, vp, i, i, sz, i, i] + [vp] * 11, i),
        "fabf_sharpen_maps": ([vp, vp, i, i, sz, C.POINTER(SharpenCfg), vp, vp, vp], i),
        "fabf_texture_sigma": ([vp, vp, i, i, sz, C.POINTER(TextureCfg), vp, vp], i),
        "fabf_sharpen": ([vp, vp, i, i, sz, C.POINTER(SharpenCfg), vp, i, vp], i),
        "fabf_texture_filter": ([vp, vp, i, i, sz, C.POINTER(TextureCfg), vp, i, vp], i),
        "fabf_luma": ([vp, vp, i, i, sz, vp, sz, vp], i),
        "fabf_filter_rgb": ([vp, vp, vp, vp, i, i, sz, i, i, vp, i, vp], i),
        "fabf_texture_filter_rgb": ([vp, vp, i, i, sz, C.POINTER(TextureCfg), vp, i, vp], i),
        "fabf_pipe_peaks": ([C.POINTER(C.c_double)], i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def status_str(status: int) -> str:
    try:
        return load().fabf_status_str(int(status)).decode()
    except Exception:   # noqa: BLE001 - only used to format messages
        return "status %d" % status


def _check(rc: int, what: str) -> None:
    if rc != FABF_OK:
        raise FabfError(rc, what)


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a) -> int:
    if a is None:
        return 0
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError("expected a torch tensor or numpy array, got %r" % type(a))


def _check_out(out, H: int, W: int, f64: bool) -> None:
    """The output buffer must hold H x W elements of the type out_is_f64 names
    (the kernels write H x W float64 or float32 values through its pointer)."""
    if out is None:
        raise ValueError("an output buffer is required")
    if _is_torch(out):
        esize, n = out.element_size(), out.numel()
        if not out.dtype.is_floating_point:
            raise ValueError("output must be float32 or float64")
    else:
        esize, n = out.dtype.itemsize, out.size
        if out.dtype.kind != "f":
            raise ValueError("output must be float32 or float64")
    if esize != (8 if f64 else 4):
        raise ValueError("output element size %d does not match out_is_f64=%s" % (esize, f64))
    if n < H * W:
        raise ValueError("output holds %d elements, %d needed" % (n, H * W))


def _check_inputs(img, theta, sigma, H: int, W: int, pitch: int) -> None:
    """img must be uint8 with at least (H-1) pitch + W bytes; theta and sigma
    float32 with H x W elements (what the kernels read through the pointers)."""
    def info(a):
        if _is_torch(a):
            return a.element_size(), a.numel(), str(a.dtype)
        return a.dtype.itemsize, a.size, str(a.dtype)
    e, n, dt = info(img)
    if e != 1 or "uint8" not in dt:
        raise ValueError("img must be uint8, got %s" % dt)
    if pitch < W or n < (H - 1) * pitch + W:
        raise ValueError("img holds %d bytes, (H-1)*pitch+W = %d needed" % (n, (H - 1) * pitch + W))
    for name, a in (("theta", theta), ("sigma", sigma)):
        e, n, dt = info(a)
        if "float32" not in dt:
            raise ValueError("%s must be float32, got %s" % (name, dt))
        if n < H * W:
            raise ValueError("%s holds %d elements, %d needed" % (name, n, H * W))


def _stream_of(*arrays) -> int:
    for a in arrays:
        if _is_torch(a) and a.is_cuda:
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return 0


def _empty_like_out(ref, H, W, f64):
    if _is_torch(ref):
        import torch
        return torch.empty((H, W), dtype=torch.float64 if f64 else torch.float32, device=ref.device)
    return np.empty((H, W), dtype=np.float64 if f64 else np.float32)


class Context:
    """``fabf_ctx``: one GPU, one default precision."""

    def __init__(self, device: int = 0, precision: int = FABF_FP64, mem_budget_bytes: int = 0,
                 autotune: int = 0, tune_cache_path: str | None = None):
        lib = load()
        cfg = _Config(device, mem_budget_bytes, precision, autotune,
                      tune_cache_path.encode() if tune_cache_path else None)
        h = C.c_void_p()
        _check(lib.fabf_create(C.byref(cfg), C.byref(h)), "fabf_create")
        self._h = h
        self.device = device

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().fabf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:   # noqa: BLE001 - interpreter shutdown
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def fabf_set_precision(ctx: Context, precision: int) -> None:
    _check(load().fabf_set_precision(ctx.handle, int(precision)), "fabf_set_precision")


def fabf_filter(ctx: Context, img, theta, sigma, w: int, N: int, out=None, out_is_f64: bool = True,
                pitch: int | None = None, stream: int | None = None, check: bool = True):
    """Algorithm 1 on one image (``fabf_filter``); returns ``out``.

    ``img`` is (H, W) uint8, or (H, pitch) with ``pitch`` given and the image
    in its first W columns (then pass W via theta's shape).
    """
    H, W = int(theta.shape[0]), int(theta.shape[1])
    p = int(pitch) if pitch is not None else int(img.shape[1])
    if out is None:
        out = _empty_like_out(theta, H, W, out_is_f64)
    _check_out(out, H, W, out_is_f64)
    _check_inputs(img, theta, sigma, H, W, p)
    s = _stream_of(img, theta, sigma, out) if stream is None else stream
    rc = load().fabf_filter(ctx.handle, _ptr(img), _ptr(theta), _ptr(sigma), H, W, p, int(w), int(N),
                            _ptr(out), 1 if out_is_f64 else 0, s)
    if check:
        _check(rc, "fabf_filter")
        return out
    return out, rc


def fabf_filter_noalloc(img, theta, sigma, w: int, N: int, out, out_is_f64: bool = True,
                        pitch: int | None = None, stream: int | None = None):
    """``fabf_filter_noalloc``: no context, device tensors only, blocking.
    Returns (status, n_fallback)."""
    H, W = int(theta.shape[0]), int(theta.shape[1])
    p = int(pitch) if pitch is not None else int(img.shape[1])
    _check_out(out, H, W, out_is_f64)
    _check_inputs(img, theta, sigma, H, W, p)
    s = _stream_of(img, theta, sigma, out) if stream is None else stream
    nf = C.c_uint64(0)
    lib = load()
    args = (_ptr(img), _ptr(theta), _ptr(sigma), H, W, p, int(w), int(N), _ptr(out), 1 if out_is_f64 else 0, s,
            C.byref(nf))
    dev = next((a.device for a in (img, theta, sigma, out) if _is_torch(a) and a.is_cuda), None)
    if dev is not None:
        import torch
        with torch.cuda.device(dev):       # the call runs on its current device
            rc = lib.fabf_filter_noalloc(*args)
    else:
        rc = lib.fabf_filter_noalloc(*args)
    return rc, nf.value


def fabf_get_status(ctx: Context, stream: int = 0):
    """(status, n_fallback) of the stream-ordered calls since the last query."""
    st = C.c_int(0)
    nf = C.c_uint64(0)
    _check(load().fabf_get_status(ctx.handle, stream, C.byref(st), C.byref(nf)), "fabf_get_status")
    return st.value, nf.value


def fabf_get_status_ex(ctx: Context, stream: int = 0):
    """(status, n_fallback, n_fp64_redo) of the stream-ordered calls since the
    last query."""
    st = C.c_int(0)
    nf = C.c_uint64(0)
    nr = C.c_uint64(0)
    _check(load().fabf_get_status_ex(ctx.handle, stream, C.byref(st), C.byref(nf), C.byref(nr)),
           "fabf_get_status_ex")
    return st.value, nf.value, nr.value


def fabf_hilbert_inverse(N: int) -> np.ndarray:
    out = np.zeros((N + 1, N + 1), dtype=np.int64)
    _check(load().fabf_hilbert_inverse(int(N), out.ctypes.data), "fabf_hilbert_inverse")
    return out


def fabf_centred_inverse(N: int) -> np.ndarray:
    out = np.zeros((N + 1, N + 1), dtype=np.float64)
    _check(load().fabf_centred_inverse(int(N), out.ctypes.data), "fabf_centred_inverse")
    return out


def fabf_fused_smem_bytes(w: int, N: int) -> int:
    b = C.c_size_t(0)
    _check(load().fabf_fused_smem_bytes(int(w), int(N), C.byref(b)), "fabf_fused_smem_bytes")
    return b.value


def fabf_debug_stages(ctx: Context, img, theta, sigma, w: int, N: int):
    """Every intermediate of Algorithm 1 (device tensors in, dict of tensors out)."""
    import torch
    H, W = int(theta.shape[0]), int(theta.shape[1])
    dev = theta.device
    o = dict(
        alpha=torch.zeros((H, W), dtype=torch.uint8, device=dev),
        beta=torch.zeros((H, W), dtype=torch.uint8, device=dev),
        m=torch.zeros((N + 1, H, W), dtype=torch.int64, device=dev),
        M=torch.zeros((N + 1, H, W), dtype=torch.int64, device=dev),
        mu=torch.full((N + 1, H, W), float("nan"), dtype=torch.float64, device=dev),
        c=torch.full((N + 1, H, W), float("nan"), dtype=torch.float64, device=dev),
        t0lam=torch.full((2, H, W), float("nan"), dtype=torch.float64, device=dev),
        I=torch.full((N + 2, H, W), float("nan"), dtype=torch.float64, device=dev),
        T=torch.full((2, H, W), float("nan"), dtype=torch.float64, device=dev),
        flags=torch.zeros((H, W), dtype=torch.int32, device=dev),
        out=torch.zeros((H, W), dtype=torch.float64, device=dev),
    )
    rc = load().fabf_debug_stages(ctx.handle, _ptr(img), _ptr(theta), _ptr(sigma), H, W,
                                  int(img.shape[1]), int(w), int(N),
                                  *[_ptr(o[k]) for k in ("alpha", "beta", "m", "M", "mu", "c",
                                                         "t0lam", "I", "T", "flags", "out")])
    _check(rc, "fabf_debug_stages")
    return o


def fabf_debug_integrals(ctx: Context, lam, t0, K: int, precision: int = FABF_FP64):
    """I_0..I_K for device float64 tensors lam, t0 -> (n, K+1) float64 tensor."""
    import torch
    n = int(lam.numel())
    out = torch.empty((n, K + 1), dtype=torch.float64, device=lam.device)
    _check(load().fabf_debug_integrals(ctx.handle, _ptr(lam), _ptr(t0), n, int(K), int(precision),
                                       _ptr(out)), "fabf_debug_integrals")
    return out


def fabf_bruteforce(ctx: Context, img, theta, sigma, w: int, out=None, out_is_f64: bool = True,
                    use_f64: bool = True, stream: int | None = None):
    """Brute-force adaptive bilateral filter on the GPU (device tensors)."""
    H, W = int(theta.shape[0]), int(theta.shape[1])
    if out is None:
        out = _empty_like_out(theta, H, W, out_is_f64)
    _check_out(out, H, W, out_is_f64)
    _check_inputs(img, theta, sigma, H, W, int(img.shape[1]))
    s = _stream_of(img, theta, sigma, out) if stream is None else stream
    _check(load().fabf_bruteforce(ctx.handle, _ptr(img), _ptr(theta), _ptr(sigma), H, W,
                                  int(img.shape[1]), int(w), _ptr(out), 1 if out_is_f64 else 0,
                                  1 if use_f64 else 0, s), "fabf_bruteforce")
    return out


def _taps(taps) -> np.ndarray:
    t = np.ascontiguousarray(np.asarray(taps), dtype=np.uint32)
    if t.ndim != 1 or len(t) % 2 != 1:
        raise ValueError("taps must be a 1-D array of odd length 2r+1")
    return t


def fabf_gaussian_taps(rho: float) -> np.ndarray:
    """Integer taps of the Gaussian spatial kernel of Eq. (4) (``fabf_gaussian_taps``)."""
    buf = np.zeros(2 * 40 + 1, np.uint32)
    r = C.c_int(0)
    _check(load().fabf_gaussian_taps(float(rho), buf.ctypes.data, len(buf), C.byref(r)),
           "fabf_gaussian_taps")
    return buf[:2 * r.value + 1].copy()


def fabf_filter_sep(ctx: Context, img, theta, sigma, taps, N: int, out=None, out_is_f64: bool = True,
                    pitch: int | None = None, stream: int | None = None, check: bool = True):
    """Algorithm 1 with the separable spatial kernel taps x taps (``fabf_filter_sep``)."""
    t = _taps(taps)
    H, W = int(theta.shape[0]), int(theta.shape[1])
    p = int(pitch) if pitch is not None else int(img.shape[1])
    if out is None:
        out = _empty_like_out(theta, H, W, out_is_f64)
    _check_out(out, H, W, out_is_f64)
    _check_inputs(img, theta, sigma, H, W, p)
    s = _stream_of(img, theta, sigma, out) if stream is None else stream
    rc = load().fabf_filter_sep(ctx.handle, _ptr(img), _ptr(theta), _ptr(sigma), H, W, p, t.ctypes.data,
                                len(t) // 2, int(N), _ptr(out), 1 if out_is_f64 else 0, s)
    if check:
        _check(rc, "fabf_filter_sep")
        return out
    return out, rc


def _stage_planes(theta, N: int) -> dict:
    import torch
    H, W = int(theta.shape[0]), int(theta.shape[1])
    dev = theta.device
    return dict(
        alpha=torch.zeros((H, W), dtype=torch.uint8, device=dev),
        beta=torch.zeros((H, W), dtype=torch.uint8, device=dev),
        m=torch.zeros((N + 1, H, W, 2), dtype=torch.int64, device=dev),
        M=torch.zeros((N + 1, H, W, 2), dtype=torch.int64, device=dev),
        mu=torch.full((N + 1, H, W), float("nan"), dtype=torch.float64, device=dev),
        c=torch.full((N + 1, H, W), float("nan"), dtype=torch.float64, device=dev),
        t0lam=torch.full((2, H, W), float("nan"), dtype=torch.float64, device=dev),
        I=torch.full((N + 2, H, W), float("nan"), dtype=torch.float64, device=dev),
        T=torch.full((2, H, W), float("nan"), dtype=torch.float64, device=dev),
        flags=torch.zeros((H, W), dtype=torch.int32, device=dev),
        out=torch.zeros((H, W), dtype=torch.float64, device=dev),
    )


_STAGE_KEYS = ("alpha", "beta", "m", "M", "mu", "c", "t0lam", "I", "T", "flags", "out")


def fabf_debug_stages_sep(ctx: Context, img, theta, sigma, taps, N: int):
    """Every intermediate with the separable kernel; m and M are (N+1, H, W, 2)
    uint64 word pairs held in int64 tensors (low word first)."""
    t = _taps(taps)
    H, W = int(theta.shape[0]), int(theta.shape[1])
    o = _stage_planes(theta, N)
    rc = load().fabf_debug_stages_sep(ctx.handle, _ptr(img), _ptr(theta), _ptr(sigma), H, W,
                                      int(img.shape[1]), t.ctypes.data, len(t) // 2, int(N),
                                      *[_ptr(o[k]) for k in _STAGE_KEYS])
    _check(rc, "fabf_debug_stages_sep")
    return o


def fabf_cascade_taps(rb: int) -> np.ndarray:
    """Taps of the three-box cascade of radius rb (``fabf_cascade_taps``)."""
    buf = np.zeros(2 * 40 + 1, np.uint32)
    r = C.c_int(0)
    _check(load().fabf_cascade_taps(int(rb), buf.ctypes.data, len(buf), C.byref(r)), "fabf_cascade_taps")
    return buf[:2 * r.value + 1].copy()


def fabf_cascade_radius(rho: float) -> int:
    """The cascade radius whose variance rb (rb + 1) is nearest rho^2."""
    rb = C.c_int(0)
    _check(load().fabf_cascade_radius(float(rho), C.byref(rb)), "fabf_cascade_radius")
    return rb.value


def fabf_filter_cascade(ctx: Context, img, theta, sigma, rb: int, N: int, out=None, out_is_f64: bool = True,
                        pitch: int | None = None, stream: int | None = None, tile_rows: int = 0,
                        check: bool = True):
    """Algorithm 1 with the three-box cascade of radius rb as spatial kernel,
    O(1) per pixel in rb (``fabf_filter_cascade``)."""
    H, W = int(theta.shape[0]), int(theta.shape[1])
    p = int(pitch) if pitch is not None else int(img.shape[1])
    if out is None:
        out = _empty_like_out(theta, H, W, out_is_f64)
    _check_out(out, H, W, out_is_f64)
    _check_inputs(img, theta, sigma, H, W, p)
    s = _stream_of(img, theta, sigma, out) if stream is None else stream
    rc = load().fabf_filter_cascade(ctx.handle, _ptr(img), _ptr(theta), _ptr(sigma), H, W, p, int(rb), int(N),
                                    _ptr(out), 1 if out_is_f64 else 0, int(tile_rows), s)
    if check:
        _check(rc, "fabf_filter_cascade")
        return out
    return out, rc


def fabf_debug_stages_cascade(ctx: Context, img, theta, sigma, rb: int, N: int):
    """fabf_debug_stages_sep's planes from the box-cascade kernel."""
    H, W = int(theta.shape[0]), int(theta.shape[1])
    o = _stage_planes(theta, N)
    rc = load().fabf_debug_stages_cascade(ctx.handle, _ptr(img), _ptr(theta), _ptr(sigma), H, W,
                                          int(img.shape[1]), int(rb), int(N), *[_ptr(o[k]) for k in _STAGE_KEYS])
    _check(rc, "fabf_debug_stages_cascade")
    return o


def fabf_debug_fp64_functions(ctx: Context, x):
    """(erfcx(|x|), exp(-|x|)) from the FP64 form's own functions, on device
    float64 tensors."""
    import torch
    e1 = torch.empty_like(x)
    e2 = torch.empty_like(x)
    _check(load().fabf_debug_fp64_functions(ctx.handle, _ptr(x), int(x.numel()), _ptr(e1), _ptr(e2)),
           "fabf_debug_fp64_functions")
    return e1, e2


def fabf_bruteforce_sep(ctx: Context, img, theta, sigma, taps, out=None, out_is_f64: bool = True,
                        use_f64: bool = True, stream: int | None = None):
    """Brute-force filter with the separable kernel on the GPU (device tensors)."""
    t = _taps(taps)
    H, W = int(theta.shape[0]), int(theta.shape[1])
    if out is None:
        out = _empty_like_out(theta, H, W, out_is_f64)
    _check_out(out, H, W, out_is_f64)
    _check_inputs(img, theta, sigma, H, W, int(img.shape[1]))
    s = _stream_of(img, theta, sigma, out) if stream is None else stream
    _check(load().fabf_bruteforce_sep(ctx.handle, _ptr(img), _ptr(theta), _ptr(sigma), H, W,
                                      int(img.shape[1]), t.ctypes.data, len(t) // 2, _ptr(out),
                                      1 if out_is_f64 else 0, 1 if use_f64 else 0, s),
           "fabf_bruteforce_sep")
    return out


def make_request(img, theta, sigma, w: int, N: int, out, out_is_f64: bool = True, passes: int = 1,
                 sigma_decay: float = 0.8, pitch: int | None = None) -> Request:
    H, W = int(theta.shape[0]), int(theta.shape[1])
    p = int(pitch) if pitch is not None else int(img.shape[1])
    _check_out(out, H, W, out_is_f64)
    _check_inputs(img, theta, sigma, H, W, p)
    return Request(_ptr(img), _ptr(theta), _ptr(sigma), H, W, p, int(w), int(N),
                   int(passes), float(sigma_decay), _ptr(out), 1 if out_is_f64 else 0)


def fabf_filter_batch(ctx: Context, reqs, stream: int = 0) -> None:
    arr = (Request * len(reqs))(*reqs)
    _check(load().fabf_filter_batch(ctx.handle, arr, len(reqs), stream), "fabf_filter_batch")


def fabf_serve_submit(ctx: Context, req: Request, check: bool = True):
    t = C.c_uint64(0)
    rc = load().fabf_serve_submit(ctx.handle, C.byref(req), C.byref(t))
    if check:
        _check(rc, "fabf_serve_submit")
        return t.value
    return rc, t.value


def fabf_serve_poll(ctx: Context, ticket: int, timeout_us: int = 0):
    """(rc, result): rc FABF_OK when done (result = the request's status),
    FABF_EAGAIN while pending, FABF_ENOTFOUND for an unknown ticket."""
    r = C.c_int(0)
    rc = load().fabf_serve_poll(ctx.handle, C.c_uint64(ticket), int(timeout_us), C.byref(r))
    return rc, r.value


def fabf_serve_stats(ctx: Context):
    """(device bytes held by admitted requests, requests still running)."""
    b = C.c_uint64(0)
    n = C.c_int(0)
    _check(load().fabf_serve_stats(ctx.handle, C.byref(b), C.byref(n)), "fabf_serve_stats")
    return b.value, n.value


def fabf_batch_stats(ctx: Context):
    """(CUDA graph captures, graph launches) of fabf_filter_batch so far."""
    c = C.c_int(0)
    n = C.c_int(0)
    _check(load().fabf_batch_stats(ctx.handle, C.byref(c), C.byref(n)), "fabf_batch_stats")
    return c.value, n.value


def fabf_tile_rows(ctx: Context, w: int, N: int, precision: int = FABF_FP64) -> int:
    """Output rows per tile used for (w, N, precision) (autotuned if enabled)."""
    t = C.c_int(0)
    _check(load().fabf_tile_rows(ctx.handle, int(w), int(N), int(precision), C.byref(t)),
           "fabf_tile_rows")
    return t.value


# ---------------------------------------------------------------------------
# Applications (Sec. IV): device tensors only
# ---------------------------------------------------------------------------
def _img_dims(img, H=None, W=None, pitch=None):
    H = int(img.shape[0]) if H is None else int(H)
    p = int(img.shape[1]) if pitch is None else int(pitch)
    W = p if W is None else int(W)
    return H, W, p


def fabf_sharpen_maps(ctx: Context, img, cfg: SharpenCfg, W=None, pitch=None, stream=None):
    """(theta, sigma) float32 maps of the sharpening rules (device tensors)."""
    import torch
    H, W, p = _img_dims(img, None, W, pitch)
    th = torch.empty((H, W), dtype=torch.float32, device=img.device)
    sg = torch.empty((H, W), dtype=torch.float32, device=img.device)
    s = _stream_of(img) if stream is None else stream
    _check(load().fabf_sharpen_maps(ctx.handle, _ptr(img), H, W, p, C.byref(cfg), _ptr(th), _ptr(sg), s),
           "fabf_sharpen_maps")
    return th, sg


def fabf_texture_sigma(ctx: Context, img, cfg: TextureCfg, W=None, pitch=None, stream=None):
    """The mRTV width map of the texture filter (float32 device tensor)."""
    import torch
    H, W, p = _img_dims(img, None, W, pitch)
    sg = torch.empty((H, W), dtype=torch.float32, device=img.device)
    s = _stream_of(img) if stream is None else stream
    _check(load().fabf_texture_sigma(ctx.handle, _ptr(img), H, W, p, C.byref(cfg), _ptr(sg), s),
           "fabf_texture_sigma")
    return sg


def fabf_sharpen(ctx: Context, img, cfg: SharpenCfg, out=None, out_is_f64: bool = True, W=None, pitch=None,
                 stream=None):
    """One sharpening pass (Sec. IV-A) on a device image."""
    H, W, p = _img_dims(img, None, W, pitch)
    if out is None:
        import torch
        out = torch.empty((H, W), dtype=torch.float64 if out_is_f64 else torch.float32, device=img.device)
    _check_out(out, H, W, out_is_f64)
    s = _stream_of(img, out) if stream is None else stream
    _check(load().fabf_sharpen(ctx.handle, _ptr(img), H, W, p, C.byref(cfg), _ptr(out), 1 if out_is_f64 else 0, s),
           "fabf_sharpen")
    return out


def fabf_texture_filter(ctx: Context, img, cfg: TextureCfg, out=None, out_is_f64: bool = True, W=None,
                        pitch=None, stream=None):
    """The texture-filtering pipeline (Sec. IV-C) on a device image."""
    H, W, p = _img_dims(img, None, W, pitch)
    if out is None:
        import torch
        out = torch.empty((H, W), dtype=torch.float64 if out_is_f64 else torch.float32, device=img.device)
    _check_out(out, H, W, out_is_f64)
    s = _stream_of(img, out) if stream is None else stream
    _check(load().fabf_texture_filter(ctx.handle, _ptr(img), H, W, p, C.byref(cfg), _ptr(out),
                                      1 if out_is_f64 else 0, s), "fabf_texture_filter")
    return out


# ---------------------------------------------------------------------------
# Colour images (Sec. IV-C): interleaved (H, W, 3) uint8 device tensors
# ---------------------------------------------------------------------------
def _rgb_dims(rgb):
    import torch
    if len(rgb.shape) != 3 or int(rgb.shape[2]) != 3 or rgb.dtype != torch.uint8:
        raise ValueError("rgb must be a uint8 tensor of shape (H, W, 3)")
    if not rgb.is_contiguous():
        raise ValueError("rgb must be contiguous")
    H, W = int(rgb.shape[0]), int(rgb.shape[1])
    return H, W, 3 * W


def _rgb_out(rgb, out, out_is_f64):
    import torch
    H, W, _ = _rgb_dims(rgb)
    dt = torch.float64 if out_is_f64 else torch.float32
    if out is None:
        return torch.empty((H, W, 3), dtype=dt, device=rgb.device)
    if tuple(out.shape) != (H, W, 3) or out.dtype != dt or not out.is_contiguous():
        raise ValueError("out must be a contiguous (H, W, 3) %s tensor" % dt)
    return out


def fabf_luma(ctx: Context, rgb, stream=None):
    """The integer BT.601 luma of an interleaved colour image (uint8 H x W)."""
    import torch
    H, W, p = _rgb_dims(rgb)
    Y = torch.empty((H, W), dtype=torch.uint8, device=rgb.device)
    s = _stream_of(rgb) if stream is None else stream
    _check(load().fabf_luma(ctx.handle, _ptr(rgb), H, W, p, _ptr(Y), W, s), "fabf_luma")
    return Y


def fabf_filter_rgb(ctx: Context, rgb, theta, sigma, w: int, N: int, out=None, out_is_f64: bool = True,
                    stream=None):
    """Algorithm 1 on each channel of an interleaved colour image; theta is
    (H, W, 3) float32 or None (theta_c = f_c), sigma one (H, W) float32 map."""
    H, W, p = _rgb_dims(rgb)
    import torch
    if tuple(sigma.shape) != (H, W) or sigma.dtype != torch.float32 or not sigma.is_contiguous():
        raise ValueError("sigma must be a contiguous (H, W) float32 tensor")
    if theta is not None and (tuple(theta.shape) != (H, W, 3) or theta.dtype != torch.float32
                              or not theta.is_contiguous()):
        raise ValueError("theta must be a contiguous (H, W, 3) float32 tensor")
    out = _rgb_out(rgb, out, out_is_f64)
    s = _stream_of(rgb, out) if stream is None else stream
    _check(load().fabf_filter_rgb(ctx.handle, _ptr(rgb), _ptr(theta), _ptr(sigma), H, W,
                                  p, w, N, _ptr(out), 1 if out_is_f64 else 0, s), "fabf_filter_rgb")
    return out


def fabf_texture_filter_rgb(ctx: Context, rgb, cfg: TextureCfg, out=None, out_is_f64: bool = True, stream=None):
    """The texture-filtering pipeline (Sec. IV-C) on an interleaved colour image."""
    H, W, p = _rgb_dims(rgb)
    out = _rgb_out(rgb, out, out_is_f64)
    s = _stream_of(rgb, out) if stream is None else stream
    _check(load().fabf_texture_filter_rgb(ctx.handle, _ptr(rgb), H, W, p, C.byref(cfg), _ptr(out),
                                          1 if out_is_f64 else 0, s), "fabf_texture_filter_rgb")
    return out


def fabf_pipe_peaks(device: int = 0) -> dict:
    """``fabf_pipe_peaks``: this GPU's measured arithmetic pipe peaks."""
    import torch
    out = (C.c_double * 6)()
    with torch.cuda.device(device):
        _check(load().fabf_pipe_peaks(out), "fabf_pipe_peaks")
    return {"fp64_tflops": out[0], "fp32_tflops": out[1], "int32_tops": out[2], "mufu_tops": out[3],
            "sm_mhz": out[4], "sms": int(out[5])}
