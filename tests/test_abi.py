"""The C-ABI library builds, loads and exports every symbol include/fabf.h
declares; host-side logic that needs no GPU (no compute calls here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest
import scipy.linalg

from paper_1811_02308_gb300 import build, fabf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return fabf.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fabf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fabf_\w+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for n in ("fabf_create", "fabf_destroy", "fabf_filter", "fabf_filter_batch",
              "fabf_serve_submit", "fabf_serve_poll", "fabf_status_str"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_library_is_built_for_sm_103a():
    # the build passes exactly one -gencode for sm_103a
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


@pytest.mark.parametrize("N", range(7))
def test_kernel_hilbert_table_is_exact(lib, N):
    got = fabf.fabf_hilbert_inverse(N)
    ref = scipy.linalg.invhilbert(N + 1, exact=True)
    assert got.tolist() == [[int(v) for v in row] for row in ref]


@pytest.mark.parametrize("N", range(7))
def test_kernel_centred_table_is_the_exact_inverse(lib, N):
    """The centred fit's table times the matrix of centred moments,
    A~[j][k] = 1/(j+k+1) for j+k even else 0, is the identity in exact
    rational arithmetic (every entry a dyadic rational held exactly)."""
    from fractions import Fraction
    got = fabf.fabf_centred_inverse(N)
    inv = [[Fraction(float(v)) for v in row] for row in got]
    A = [[Fraction(1, j + k + 1) if (j + k) % 2 == 0 else Fraction(0) for k in range(N + 1)]
         for j in range(N + 1)]
    for i in range(N + 1):
        for k in range(N + 1):
            assert sum(inv[i][j] * A[j][k] for j in range(N + 1)) == (1 if i == k else 0)
    # the checkerboard: even and odd coefficients do not mix
    for i in range(N + 1):
        for k in range(N + 1):
            if (i + k) % 2:
                assert got[i][k] == 0.0


def test_argument_checks_without_gpu(lib):
    null = C.c_void_p(0)
    assert lib.fabf_filter(null, 0, 0, 0, 4, 4, 4, 1, 1, 0, 1, 0) == fabf.FABF_EINVAL
    out = np.zeros(64, np.int64)
    assert lib.fabf_hilbert_inverse(7, out.ctypes.data) == fabf.FABF_EUNSUPPORTED
    assert lib.fabf_hilbert_inverse(3, None) == fabf.FABF_EINVAL
    assert lib.fabf_centred_inverse(7, np.zeros(64).ctypes.data) == fabf.FABF_EUNSUPPORTED
    assert lib.fabf_centred_inverse(3, None) == fabf.FABF_EINVAL
    b = C.c_size_t(0)
    assert lib.fabf_fused_smem_bytes(41, 5, C.byref(b)) == fabf.FABF_EUNSUPPORTED
    assert lib.fabf_fused_smem_bytes(5, 7, C.byref(b)) == fabf.FABF_EUNSUPPORTED
    assert lib.fabf_fused_smem_bytes(0, 5, C.byref(b)) == fabf.FABF_EINVAL
    assert lib.fabf_create(None, None) == fabf.FABF_EINVAL


def test_shared_memory_fits_two_ctas_per_sm(lib):
    # 227 KB per SM: two resident CTAs need <= 113 KB each, for every (w, N)
    worst = max(fabf.fabf_fused_smem_bytes(w, N) for w in range(1, 41) for N in range(7))
    assert worst <= 113 * 1024


def test_status_strings(lib):
    for s in range(8):
        assert fabf.status_str(s)
    assert "unknown" in fabf.status_str(99)


def test_gaussian_taps_helper_matches_the_input_generator(lib):
    from paper_1811_02308_gb300 import synth
    for rho in (0.2, 0.5, 1.0, 1.7, 3.0, 5.0, 7.5, 10.0, 13.0, 40.0 / 3.0):
        assert np.array_equal(fabf.fabf_gaussian_taps(rho), synth.gaussian_taps(rho)), rho


def test_separable_argument_checks_without_gpu(lib):
    buf = np.zeros(81, np.uint32)
    r = C.c_int(0)
    assert lib.fabf_gaussian_taps(0.0, buf.ctypes.data, 81, C.byref(r)) == fabf.FABF_EINVAL
    assert lib.fabf_gaussian_taps(float("nan"), buf.ctypes.data, 81, C.byref(r)) == fabf.FABF_EINVAL
    assert lib.fabf_gaussian_taps(13.4, buf.ctypes.data, 81, C.byref(r)) == fabf.FABF_EUNSUPPORTED
    assert lib.fabf_gaussian_taps(3.0, buf.ctypes.data, 18, C.byref(r)) == fabf.FABF_EINVAL
    null = C.c_void_p(0)
    assert lib.fabf_filter_sep(null, 0, 0, 0, 4, 4, 4, buf.ctypes.data, 1, 1, 0, 1, 0) == fabf.FABF_EINVAL


def test_cascade_taps_are_the_three_fold_box_convolution(lib):
    for rb in range(1, 14):
        box = np.ones(2 * rb + 1, np.int64)
        ref = np.convolve(np.convolve(box, box), box)
        t = fabf.fabf_cascade_taps(rb)
        assert len(t) == 6 * rb + 1 and np.array_equal(t.astype(np.int64), ref), rb
        assert int(t.sum()) == (2 * rb + 1) ** 3
        # the variance of a sum of three independent uniform variables on
        # {-rb..rb}: 3 (n^2 - 1) / 12 = rb (rb + 1), exactly
        d = np.arange(-3 * rb, 3 * rb + 1)
        assert int((t.astype(np.int64) * d * d).sum()) == rb * (rb + 1) * int(t.sum())


def test_cascade_radius_and_argument_checks_without_gpu(lib):
    for rho in (0.3, 1.0, 1.5, 2.4, 3.0, 5.0, 7.7, 10.0, 13.0, 13.6):
        rb = fabf.fabf_cascade_radius(rho)
        best = min(range(1, 14), key=lambda k: abs(k * (k + 1) - rho * rho))
        assert rb == best, rho
    buf = np.zeros(81, np.uint32)
    r = C.c_int(0)
    rb = C.c_int(0)
    assert lib.fabf_cascade_radius(0.0, C.byref(rb)) == fabf.FABF_EINVAL
    assert lib.fabf_cascade_radius(float("inf"), C.byref(rb)) == fabf.FABF_EINVAL
    assert lib.fabf_cascade_radius(14.5, C.byref(rb)) == fabf.FABF_EUNSUPPORTED
    assert lib.fabf_cascade_taps(0, buf.ctypes.data, 81, C.byref(r)) == fabf.FABF_EINVAL
    assert lib.fabf_cascade_taps(14, buf.ctypes.data, 81, C.byref(r)) == fabf.FABF_EUNSUPPORTED
    assert lib.fabf_cascade_taps(3, buf.ctypes.data, 18, C.byref(r)) == fabf.FABF_EINVAL
    null = C.c_void_p(0)
    assert lib.fabf_filter_cascade(null, 0, 0, 0, 4, 4, 4, 1, 1, 0, 1, 0, 0) == fabf.FABF_EINVAL
    assert lib.fabf_filter_cascade(null, 0, 0, 0, 4, 4, 4, 1, 1, 0, 1, 12, 0) == fabf.FABF_EINVAL
    assert lib.fabf_filter_cascade(null, 0, 0, 0, 4, 4, 4, 14, 1, 0, 1, 0, 0) == fabf.FABF_EUNSUPPORTED


def test_binding_rejects_mismatched_buffers():
    # the binding checks buffer types and sizes before any pointer reaches
    # a kernel (a float32 output passed with out_is_f64 = True would be
    # written past its end)
    H, W = 4, 6
    img = np.zeros((H, W), np.uint8)
    th = np.zeros((H, W), np.float32)
    fabf._check_out(np.zeros((H, W), np.float64), H, W, True)
    fabf._check_out(np.zeros((H, W), np.float32), H, W, False)
    fabf._check_inputs(img, th, th, H, W, W)
    bad_out = [(np.zeros((H, W), np.float32), True), (np.zeros((H, W), np.float64), False),
               (np.zeros((H, W - 1), np.float64), True), (np.zeros((H, W), np.int64), True)]
    for out, f64 in bad_out:
        with pytest.raises(ValueError):
            fabf._check_out(out, H, W, f64)
    bad_in = [(np.zeros((H, W), np.int8), th, th, W), (img, th.astype(np.float64), th, W),
              (img, th, th[:, :-1], W), (img, th, th, W + 1), (img, th, th, W - 1)]
    for a, b, c, p in bad_in:
        with pytest.raises(ValueError):
            fabf._check_inputs(a, b, c, H, W, p)


def test_precision_enum_bounds_without_gpu(lib):
    # fabf_create checks the precision before touching the device
    h = C.c_void_p()
    cfg = fabf._Config(0, 0, 4, 0, None)
    assert lib.fabf_create(C.byref(cfg), C.byref(h)) == fabf.FABF_EINVAL
    cfg = fabf._Config(0, 0, -1, 0, None)
    assert lib.fabf_create(C.byref(cfg), C.byref(h)) == fabf.FABF_EINVAL
    assert lib.fabf_set_precision(None, fabf.FABF_CFP32) == fabf.FABF_EINVAL


def test_colour_and_application_argument_checks_without_gpu(lib):
    # argument checks that return before any CUDA call
    null = C.c_void_p(0)
    buf = np.zeros(64, np.uint8)
    out = np.zeros(64, np.float64)
    assert lib.fabf_luma(null, buf.ctypes.data, 4, 4, 12, buf.ctypes.data, 4, 0) == fabf.FABF_EINVAL
    assert lib.fabf_filter_rgb(null, buf.ctypes.data, 0, out.ctypes.data, 4, 4, 12, 2, 3, out.ctypes.data, 1,
                               0) == fabf.FABF_EINVAL
    tx = fabf.TextureCfg(3, 5, 2, 1.0, 8.0, 5.0, 60.0, 0.8, fabf.SharpenCfg(3, 5, 1.0, 10.0, 10.0, 40.0))
    assert lib.fabf_texture_filter_rgb(null, buf.ctypes.data, 4, 4, 12, C.byref(tx), out.ctypes.data, 1,
                                       0) == fabf.FABF_EINVAL
    sh = fabf.SharpenCfg(3, 5, 1.0, 10.0, 10.0, 40.0)
    assert lib.fabf_sharpen(null, buf.ctypes.data, 4, 4, 4, C.byref(sh), out.ctypes.data, 1, 0) == fabf.FABF_EINVAL
    assert lib.fabf_texture_filter(null, buf.ctypes.data, 4, 4, 4, C.byref(tx), out.ctypes.data, 1,
                                   0) == fabf.FABF_EINVAL


def test_colour_binding_rejects_bad_shapes():
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        fabf._rgb_dims(torch.zeros((4, 4, 2), dtype=torch.uint8))
    with pytest.raises(ValueError):
        fabf._rgb_dims(torch.zeros((4, 4, 3), dtype=torch.float32))
    assert fabf._rgb_dims(torch.zeros((4, 5, 3), dtype=torch.uint8)) == (4, 5, 15)
