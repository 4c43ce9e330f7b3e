"""Parity of the box-cascade CUDA path (fabf_filter_cascade: the spatial
kernel t x t, t = three-fold convolution of a box of length 2 rb + 1, summed
in O(1) per pixel) with the CPU oracle's separable path on the same taps.

The taps the oracle gets are built here with numpy (np.convolve of ones), not
by the library.  Bar: alpha, beta, the weighted moments m_k and M_k
(128-bit integers) bit-exact; mu_k, c, t0, lambda bit-exact; I_k within
1e-12 relative; the output within 1e-9 relative (floor 1 gray level).  The
cascade must also equal the direct-FIR separable path on the same taps bit
for bit in every precision form, at every tile height."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1811_02308_gb300 import build, fabf, synth  # noqa: E402

pytestmark = pytest.mark.gpu

RTOL_G = 1e-9
FORMS = [fabf.FABF_FP64, fabf.FABF_FP64FIT_FP32REC, fabf.FABF_CFP32, fabf.FABF_C32]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    c = fabf.Context(device=0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def g_err(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)
    return float(err.max()) if err.size else 0.0


def inputs(H, W, seed, n_blobs=20):
    return synth.make_inputs(H, W, seed, n_blobs=n_blobs, zeta_range=(-20, 20), sigma_range=(5, 60))


def words_to_int(a):
    a = np.asarray(a).view(np.uint64)
    return a[..., 0].astype(object) + (a[..., 1].astype(object) << 64)


def cascade_taps(rb):
    box = np.ones(2 * rb + 1, np.int64)
    return np.convolve(np.convolve(box, box), box).astype(np.uint32)


STAGE_CASES = [
    # H, W, rb, N, seed
    (1, 1, 1, 5, 1),
    (1, 77, 2, 4, 2),
    (53, 1, 1, 6, 3),
    (67, 131, 1, 5, 4),      # several tiles, ragged tails
    (67, 131, 3, 6, 5),
    (70, 150, 5, 3, 6),
    (40, 70, 13, 5, 7),      # r = 39: window larger than the image
    (33, 65, 1, 0, 8),
    (96, 200, 4, 2, 9),
    (130, 170, 13, 6, 10),   # largest radius and degree
]


@pytest.mark.parametrize("H,W,rb,N,seed", STAGE_CASES)
def test_cascade_stages_match_oracle(ctx, oracle_mod, H, W, rb, N, seed):
    f, th, s = inputs(H, W, seed)
    taps = cascade_taps(rb)
    r = len(taps) // 2
    o = fabf.fabf_debug_stages_cascade(ctx, dev(f), dev(th), dev(s), rb, N)
    a_ref, b_ref = oracle_mod.bounds(f, r)
    assert np.array_equal(o["alpha"].cpu().numpy(), a_ref)
    assert np.array_equal(o["beta"].cpu().numpy(), b_ref)
    m_ref = oracle_mod.moments_sep(f, taps, N)
    assert (words_to_int(o["m"].cpu().numpy()) == m_ref).all()
    flat = a_ref == b_ref
    flags = o["flags"].cpu().numpy()
    assert np.array_equal((flags & 1) != 0, flat)
    M = words_to_int(o["M"].cpu().numpy())
    mu, c = o["mu"].cpu().numpy(), o["c"].cpu().numpy()
    t0lam, I = o["t0lam"].cpu().numpy(), o["I"].cpu().numpy()
    out = o["out"].cpu().numpy()
    ys, xs = np.nonzero(~flat)
    rng = np.random.default_rng(seed)
    if len(ys) > 300:
        pick = rng.choice(len(ys), 300, replace=False)
        ys, xs = ys[pick], xs[pick]
    for y, x in zip(ys, xs):
        tr = oracle_mod.fabf_sep_trace(f, th, s, taps, N, y, x)
        assert list(M[:, y, x]) == tr["M"], (y, x)
        assert np.array_equal(mu[:, y, x], tr["mu"]), (y, x)
        assert np.array_equal(c[:, y, x], tr["c"]), (y, x)
        assert t0lam[0, y, x] == tr["t0"] and t0lam[1, y, x] == tr["lam"]
        np.testing.assert_allclose(I[:, y, x], tr["I"], rtol=1e-12, atol=0)
        assert bool(flags[y, x] & 2) == tr["fallback"], (y, x)
    g_ref, _ = oracle_mod.fabf_sep(f, th, s, taps, N)
    assert g_err(out, g_ref) <= RTOL_G


@pytest.mark.parametrize("prec", FORMS)
@pytest.mark.parametrize("rb,N", [(1, 5), (3, 6), (6, 4), (13, 5), (2, 0), (1, 2), (9, 3)])
def test_cascade_equals_fir_bit_for_bit(ctx, prec, rb, N):
    # both paths sum exact integer moments, so the results agree in every bit
    f, th, s = inputs(150, 233, 100 + rb)
    d = [dev(a) for a in (f, th, s)]
    taps = cascade_taps(rb)
    fabf.fabf_set_precision(ctx, prec)
    try:
        for f64 in (True, False):
            a = fabf.fabf_filter_cascade(ctx, *d, rb, N, out_is_f64=f64)
            b = fabf.fabf_filter_sep(ctx, *d, taps, N, out_is_f64=f64)
            torch.cuda.synchronize()
            assert torch.equal(a, b), (prec, rb, N, f64)
        st, _ = fabf.fabf_get_status(ctx)
    finally:
        fabf.fabf_set_precision(ctx, fabf.FABF_FP64)
    assert st == fabf.FABF_OK


@pytest.mark.parametrize("prec", [fabf.FABF_FP64, fabf.FABF_C32])
def test_cascade_tile_heights_give_identical_bits(ctx, prec):
    f, th, s = inputs(203, 301, 55)
    d = [dev(a) for a in (f, th, s)]
    fabf.fabf_set_precision(ctx, prec)
    try:
        for rb in (2, 9):
            outs = [fabf.fabf_filter_cascade(ctx, *d, rb, 5, tile_rows=t) for t in (0, 8, 16, 40, 64)]
            torch.cuda.synchronize()
            assert all(torch.equal(outs[0], o) for o in outs[1:]), rb
    finally:
        fabf.fabf_set_precision(ctx, fabf.FABF_FP64)


@pytest.mark.parametrize("rb,N", [(2, 5), (5, 5), (13, 6)])
def test_cascade_full_size_sampled(ctx, oracle_mod, rb, N):
    # 1920 x 1080 frame: every pixel on the GPU in the FP64 and centred
    # binary32 forms, 2500 sampled pixels (and the corners) by the oracle
    H, W = 1080, 1920
    f, th, s = inputs(H, W, 1001, n_blobs=200)
    taps = cascade_taps(rb)
    d = [dev(a) for a in (f, th, s)]
    g64 = fabf.fabf_filter_cascade(ctx, *d, rb, N).cpu().numpy()
    st, _ = fabf.fabf_get_status(ctx)
    assert st == fabf.FABF_OK
    fabf.fabf_set_precision(ctx, fabf.FABF_C32)
    try:
        g32 = fabf.fabf_filter_cascade(ctx, *d, rb, N, out_is_f64=False).cpu().numpy()
        st, _ = fabf.fabf_get_status(ctx)
    finally:
        fabf.fabf_set_precision(ctx, fabf.FABF_FP64)
    assert st == fabf.FABF_OK
    rng = np.random.default_rng(rb)
    ys = np.concatenate([rng.integers(0, H, 2500), [0, 0, H - 1, H - 1]])
    xs = np.concatenate([rng.integers(0, W, 2500), [0, W - 1, 0, W - 1]])
    ref, _ = oracle_mod.fabf_sep_pixels(f, th, s, taps, N, ys, xs)
    assert g_err(g64[ys, xs], ref) <= RTOL_G
    err = np.abs(g32[ys, xs].astype(np.float64) - ref)
    assert float(err.max()) <= 0.3 and float(np.sqrt(np.mean(err * err))) <= 0.01


def test_cascade_host_buffers_unaligned_pitch_and_status(ctx, oracle_mod):
    f, th, s = inputs(45, 99, 77)
    rb = 3
    ref, _ = oracle_mod.fabf_sep(f, th, s, cascade_taps(rb), 5)
    # host (pageable) buffers, float32 output
    out = np.zeros((45, 99), np.float32)
    fabf.fabf_filter_cascade(ctx, f, th, s, rb, 5, out=out, out_is_f64=False)
    assert float(np.max(np.abs(out.astype(np.float64) - ref))) <= 1e-4 * 255
    # a pitch that is not a multiple of 16 takes the plain tile load
    pitch = 101
    buf = np.zeros((45, pitch), np.uint8)
    buf[:, :99] = f
    g = fabf.fabf_filter_cascade(ctx, dev(buf), dev(th), dev(s), rb, 5, pitch=pitch).cpu().numpy()
    assert g_err(g, ref) <= RTOL_G
    # a constant image comes back exactly; a non-positive sigma sets the status
    c = np.full((40, 70), 93, np.uint8)
    gc = fabf.fabf_filter_cascade(ctx, dev(c), dev(c.astype(np.float32)), dev(np.full((40, 70), 9, np.float32)),
                                  4, 5).cpu().numpy()
    assert np.array_equal(gc, c.astype(np.float64))
    s2 = s.copy()
    s2[3, 4] = 0.0
    _, rc = fabf.fabf_filter_cascade(ctx, f, th, s2, rb, 5, check=False)
    assert rc == fabf.FABF_EINVAL


@pytest.mark.parametrize("H,W,rb,N", [(65535, 9, 13, 6), (5, 65535, 13, 5), (65535, 3, 1, 3)])
def test_cascade_maximum_dimensions(ctx, oracle_mod, H, W, rb, N):
    # the largest height / width the ABI accepts, every pixel computed in the
    # FP64 and centred forms, sampled pixels (and the corners) by the oracle
    f, th, s = inputs(H, W, 950 + W, n_blobs=10)
    taps = cascade_taps(rb)
    d = [dev(a) for a in (f, th, s)]
    g64 = fabf.fabf_filter_cascade(ctx, *d, rb, N).cpu().numpy()
    st, _ = fabf.fabf_get_status(ctx)
    assert st == fabf.FABF_OK
    fabf.fabf_set_precision(ctx, fabf.FABF_C32)
    try:
        g32 = fabf.fabf_filter_cascade(ctx, *d, rb, N, out_is_f64=False).cpu().numpy()
        st, _ = fabf.fabf_get_status(ctx)
    finally:
        fabf.fabf_set_precision(ctx, fabf.FABF_FP64)
    assert st == fabf.FABF_OK
    rng = np.random.default_rng(H + W + rb)
    ys = np.concatenate([rng.integers(0, H, 1200), [0, 0, H - 1, H - 1]])
    xs = np.concatenate([rng.integers(0, W, 1200), [0, W - 1, 0, W - 1]])
    ref, _ = oracle_mod.fabf_sep_pixels(f, th, s, taps, N, ys, xs)
    assert g_err(g64[ys, xs], ref) <= RTOL_G
    assert float(np.max(np.abs(g32[ys, xs].astype(np.float64) - ref))) <= 0.3
    assert np.isfinite(g64).all() and np.isfinite(g32).all()


@pytest.mark.parametrize("prec", FORMS)
def test_cascade_pinned_host_buffers_equal_device_path(ctx, prec):
    # pinned theta, sigma and out are read and written in place by the kernel
    # (only the image is copied): the result equals the device-pointer call
    f, th, s = inputs(130, 210, 61)
    fabf.fabf_set_precision(ctx, prec)
    try:
        for f64 in (True, False):
            dref = fabf.fabf_filter_cascade(ctx, dev(f), dev(th), dev(s), 4, 5, out_is_f64=f64).cpu().numpy()
            img = torch.from_numpy(f).pin_memory()
            pth = torch.from_numpy(th).pin_memory()
            psg = torch.from_numpy(s).pin_memory()
            pout = torch.empty((130, 210), dtype=torch.float64 if f64 else torch.float32).pin_memory()
            fabf.fabf_filter_cascade(ctx, img, pth, psg, 4, 5, out=pout, out_is_f64=f64)
            assert np.array_equal(pout.numpy(), dref), (prec, f64)
    finally:
        fabf.fabf_set_precision(ctx, fabf.FABF_FP64)
