"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: integer stages (alpha, beta, m_k, M_k) bit-exact; the FP64 shift-scale
mu_k, fit c, t0 and lambda bit-exact (same IEEE operations in the same
order on both sides); the integrals I_k within 1e-12 relative inside the
workloads' domain; the output g_hat within 1e-9 relative (floor 1 gray
level): |g_gpu - g_oracle| <= 1e-9 * max(|g_oracle|, 1)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1811_02308_gb300 import build, fabf, synth  # noqa: E402

pytestmark = pytest.mark.gpu

RTOL_G = 1e-9


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


def g_close(got, ref, rtol=RTOL_G):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)
    return float(err.max()) if err.size else 0.0


def inputs(H, W, seed, n_blobs=20, zeta=(-20, 20), sigma=(5, 60)):
    return synth.make_inputs(H, W, seed, n_blobs=n_blobs, zeta_range=zeta, sigma_range=sigma)


# ---------------------------------------------------------------------------
# Stage by stage
# ---------------------------------------------------------------------------
STAGE_CASES = [
    # H, W, w, N, seed
    (1, 1, 3, 5, 1),
    (1, 77, 4, 4, 2),
    (53, 1, 5, 6, 3),
    (3, 517, 7, 5, 4),
    (67, 131, 5, 5, 5),      # several tiles and a ragged tail in both directions
    (67, 131, 20, 6, 6),
    (40, 70, 40, 3, 7),      # window larger than the image
    (33, 65, 1, 0, 8),
    (96, 200, 13, 2, 9),
    (64, 64, 17, 1, 10),
]


def test_t0_and_lambda_are_the_correctly_rounded_quotients(ctx):
    """t0 = (theta - alpha) / d and lambda = d^2 / (2 sigma^2) (Eq. 25) in the
    FP64 form equal the IEEE binary64 quotients bit for bit, on 147k windows
    of a noise image with sigma spread over nine decades and theta over
    [-50, 300] (the kernel forms t0 from a table of correctly rounded
    reciprocals, and lambda's operands from a table of powers of d and from
    the bits of sigma)."""
    H = W = 384
    rng = np.random.default_rng(77)
    f = rng.integers(0, 256, (H, W), dtype=np.uint8)
    th = rng.uniform(-50, 300, (H, W)).astype(np.float32)
    s = (10.0 ** rng.uniform(-3, 6, (H, W))).astype(np.float32)
    s[0, :8] = [np.float32(v) for v in (1e-3, 0.1, 1.0, 5.0, 60.0, 255.0, 1e5, 1e6)]
    o = fabf.fabf_debug_stages(ctx, dev(f), dev(th), dev(s), 2, 2)
    a = o["alpha"].cpu().numpy().astype(np.float64)
    b = o["beta"].cpu().numpy().astype(np.float64)
    t0lam = o["t0lam"].cpu().numpy()
    live = b > a
    assert live.sum() > 140000
    d = (b - a)[live]
    s64 = s.astype(np.float64)[live]
    lam_ref = (d * d) / (2.0 * s64 * s64)
    t0_ref = (th.astype(np.float64)[live] - a[live]) / d
    assert np.array_equal(t0lam[1][live].view(np.uint64), lam_ref.view(np.uint64))
    assert np.array_equal(t0lam[0][live].view(np.uint64), t0_ref.view(np.uint64))


@pytest.mark.parametrize("H,W,w,N,seed", STAGE_CASES)
def test_stages_match_oracle(ctx, oracle_mod, H, W, w, N, seed):
    f, th, s = inputs(H, W, seed)
    o = fabf.fabf_debug_stages(ctx, dev(f), dev(th), dev(s), w, N)
    a_ref, b_ref = oracle_mod.bounds(f, w)
    assert np.array_equal(o["alpha"].cpu().numpy(), a_ref)
    assert np.array_equal(o["beta"].cpu().numpy(), b_ref)
    m_ref = oracle_mod.moments(f, w, N)
    assert np.array_equal(o["m"].cpu().numpy(), m_ref)
    flat = a_ref == b_ref
    M_ref = oracle_mod.shifted_moments(f, w, N)
    assert np.array_equal(o["M"].cpu().numpy()[:, ~flat], M_ref[:, ~flat])
    mu, c = o["mu"].cpu().numpy(), o["c"].cpu().numpy()
    t0lam, I, T = o["t0lam"].cpu().numpy(), o["I"].cpu().numpy(), o["T"].cpu().numpy()
    out, flags = o["out"].cpu().numpy(), o["flags"].cpu().numpy()
    assert np.array_equal((flags & 1) != 0, flat)
    ys, xs = np.nonzero(~flat)
    rng = np.random.default_rng(seed)
    if len(ys) > 600:
        pick = rng.choice(len(ys), 600, replace=False)
        ys, xs = ys[pick], xs[pick]
    for y, x in zip(ys, xs):
        tr = oracle_mod.fabf_trace(f, th, s, w, N, y, x)
        assert np.array_equal(mu[:, y, x], tr["mu"]), (y, x)
        assert np.array_equal(c[:, y, x], tr["c"]), (y, x)
        assert np.array_equal(c[:, y, x], oracle_mod.fit(N, tr["mu"])), (y, x)
        assert t0lam[0, y, x] == tr["t0"] and t0lam[1, y, x] == tr["lam"]
        np.testing.assert_allclose(I[:, y, x], tr["I"], rtol=1e-12, atol=0)
        assert bool(flags[y, x] & 2) == tr["fallback"], (y, x, T[:, y, x], tr["T1"], tr["T2"])
        assert g_close(out[y, x], tr["g"]) <= RTOL_G, (y, x, out[y, x], tr["g"])
    g_ref, _ = oracle_mod.fabf(f, th, s, w, N)
    assert g_close(out, g_ref) <= RTOL_G


# ---------------------------------------------------------------------------
# The integral engine alone, across the (lambda, t0) domain
# ---------------------------------------------------------------------------
def _grid(x_max):
    lams = np.geomspace(1e-7, 3e3, 61)
    pts = []
    for lam in lams:
        sl = np.sqrt(lam)
        xs = np.linspace(0, x_max, 7)
        t0s = list(np.linspace(0, 1, 9)) + list(-xs[1:] / sl) + list(1 + xs[1:] / sl)
        pts += [(lam, t) for t in t0s]
    return np.array(pts)


@pytest.mark.parametrize("K", [1, 4, 7])
def test_integral_engine_interior(ctx, oracle_mod, K):
    """Centre within 1.5 kernel widths of [0, 1] (x = sqrt(lambda) d <= 1.5)."""
    g = _grid(1.5)
    got = fabf.fabf_debug_integrals(ctx, dev(g[:, 0].copy()), dev(g[:, 1].copy()), K).cpu().numpy()
    for j, (lam, t0) in enumerate(g):
        ref = oracle_mod.integrals(lam, t0, K)
        np.testing.assert_allclose(got[j], ref, rtol=1e-12, atol=0, err_msg=str((lam, t0)))


def test_integral_engine_far_centre(ctx, oracle_mod):
    """Centre up to 2.83 kernel widths outside [0, 1] (the workloads' limit
    |zeta| <= 20, sigma >= 5): looser, the forward recursion loses digits
    when the centre lies far left of 0 and lambda >= 1."""
    g = _grid(2.83)
    K = 7
    got = fabf.fabf_debug_integrals(ctx, dev(g[:, 0].copy()), dev(g[:, 1].copy()), K).cpu().numpy()
    worst = 0.0
    for j, (lam, t0) in enumerate(g):
        ref = oracle_mod.integrals(lam, t0, K)
        worst = max(worst, float(np.max(np.abs(got[j] - ref) / np.abs(ref))))
    assert worst <= 5e-9, worst


# ---------------------------------------------------------------------------
# Whole images
# ---------------------------------------------------------------------------
def test_config0_full_image(ctx, oracle_mod):
    """256x256, 20 blobs, w = 5, theta = f, sigma in [10, 40], N = 5, FP64."""
    f, th, s = synth.make_inputs(256, 256, synth.config_seed(0, 0), n_blobs=20,
                                 sigma_range=(10, 40), zeta_range=None)
    g = fabf.fabf_filter(ctx, dev(f), dev(th), dev(s), 5, 5).cpu().numpy()
    st, nfb = fabf.fabf_get_status(ctx)
    g_ref, nf_ref = oracle_mod.fabf(f, th, s, 5, 5)
    assert st == fabf.FABF_OK
    assert nfb == nf_ref
    assert g_close(g, g_ref) <= RTOL_G


@pytest.mark.parametrize("w", [5, 10, 20, 40])
@pytest.mark.parametrize("N", [3, 4, 5, 6])
def test_config1_sampled(ctx, oracle_mod, w, N):
    """1920x1080, 200 blobs, theta = f + zeta, sigma in [5, 60]: every pixel on
    the GPU, a sample (borders, tile seams, random) on the oracle."""
    f, th, s = synth.make_inputs(1080, 1920, synth.config_seed(1, 0), n_blobs=200,
                                 zeta_range=(-20, 20), sigma_range=(5, 60))
    g = fabf.fabf_filter(ctx, dev(f), dev(th), dev(s), w, N).cpu().numpy()
    rng = np.random.default_rng(100 * w + N)
    ys = np.concatenate([rng.integers(0, 1080, 700), [0, 0, 1079, 1079, 31, 32, 63, 64, 540],
                         rng.integers(0, 1080, 64)])
    xs = np.concatenate([rng.integers(0, 1920, 700), [0, 1919, 0, 1919, 63, 64, 127, 128, 960],
                         np.full(64, 1919)])
    ref, _ = oracle_mod.fabf_pixels(f, th, s, w, N, ys, xs)
    assert g_close(g[ys, xs], ref) <= RTOL_G


def test_config3_size_sampled(ctx, oracle_mod):
    """4096x4096 (the largest workload), w = 20, N = 6."""
    f, th, s = synth.make_inputs(4096, 4096, synth.config_seed(3, 0), n_blobs=2000,
                                 zeta_range=None, sigma_range=(5, 60))
    g = fabf.fabf_filter(ctx, dev(f), dev(th), dev(s), 20, 6, out_is_f64=True).cpu().numpy()
    rng = np.random.default_rng(3)
    ys = np.concatenate([rng.integers(0, 4096, 400), [0, 4095, 4095, 0]])
    xs = np.concatenate([rng.integers(0, 4096, 400), [0, 4095, 0, 4095]])
    ref, _ = oracle_mod.fabf_pixels(f, th, s, 20, 6, ys, xs)
    assert g_close(g[ys, xs], ref) <= RTOL_G


# ---------------------------------------------------------------------------
# Edge cases and API paths
# ---------------------------------------------------------------------------
def test_constant_image_exact(ctx):
    f = np.full((45, 77), 201, np.uint8)
    th = f.astype(np.float32) - 7.0
    s = np.full(f.shape, 9.0, np.float32)
    g = fabf.fabf_filter(ctx, dev(f), dev(th), dev(s), 6, 5).cpu().numpy()
    assert np.array_equal(g, f.astype(np.float64))


@pytest.mark.parametrize("N", range(7))
def test_every_degree(ctx, oracle_mod, N):
    f, th, s = inputs(70, 90, 200 + N)
    g = fabf.fabf_filter(ctx, dev(f), dev(th), dev(s), 6, N).cpu().numpy()
    g_ref, _ = oracle_mod.fabf(f, th, s, 6, N)
    assert g_close(g, g_ref) <= RTOL_G


def test_unaligned_pitch_takes_plain_load_and_agrees(ctx, oracle_mod):
    """A pitch that is not a multiple of 16 bytes cannot use TMA; the plain
    shared-memory load must give the same bits as the TMA path."""
    H, W = 61, 97
    f, th, s = inputs(H, W, 300)
    buf = np.zeros((H, 101), np.uint8)
    buf[:, :W] = f
    g_plain = fabf.fabf_filter(ctx, dev(buf), dev(th), dev(s), 9, 5, pitch=101).cpu().numpy()
    buf16 = np.zeros((H, 112), np.uint8)
    buf16[:, :W] = f
    g_tma = fabf.fabf_filter(ctx, dev(buf16), dev(th), dev(s), 9, 5, pitch=112).cpu().numpy()
    assert np.array_equal(g_plain, g_tma)
    g_ref, _ = oracle_mod.fabf(f, th, s, 9, 5)
    assert g_close(g_plain, g_ref) <= RTOL_G


def test_host_pointers_and_float32_out(ctx, oracle_mod):
    f, th, s = inputs(50, 60, 400)
    g64 = fabf.fabf_filter(ctx, f, th, s, 4, 4, out_is_f64=True)     # numpy: host path
    g32 = fabf.fabf_filter(ctx, f, th, s, 4, 4, out_is_f64=False)
    g_dev = fabf.fabf_filter(ctx, dev(f), dev(th), dev(s), 4, 4).cpu().numpy()
    assert isinstance(g64, np.ndarray) and g32.dtype == np.float32
    assert np.array_equal(g64, g_dev)
    assert np.array_equal(g32, g_dev.astype(np.float32))


def test_bad_sigma_is_reported(ctx):
    f, th, s = inputs(20, 30, 500)
    s = s.copy()
    s[3, 4] = 0.0
    s[5, 6] = np.nan
    out, rc = fabf.fabf_filter(ctx, f, th, s, 3, 3, check=False)
    assert rc == fabf.FABF_EINVAL
    assert np.isnan(out[3, 4]) and np.isnan(out[5, 6])
    assert np.isfinite(np.delete(out.ravel(), [3 * 30 + 4, 5 * 30 + 6])).all()


def test_argument_errors(ctx):
    f, th, s = inputs(8, 8, 600)
    for w, N, want in [(0, 3, fabf.FABF_EINVAL), (41, 3, fabf.FABF_EUNSUPPORTED),
                       (3, 7, fabf.FABF_EUNSUPPORTED), (3, -1, fabf.FABF_EINVAL)]:
        _, rc = fabf.fabf_filter(ctx, f, th, s, w, N, check=False)
        assert rc == want


# ---------------------------------------------------------------------------
# GPU brute force (the comparator)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("w", [1, 5, 12])
def test_bruteforce_matches_oracle(ctx, oracle_mod, w):
    f, th, s = inputs(41, 83, 700 + w)
    g64 = fabf.fabf_bruteforce(ctx, dev(f), dev(th), dev(s), w, use_f64=True).cpu().numpy()
    g32 = fabf.fabf_bruteforce(ctx, dev(f), dev(th), dev(s), w, use_f64=False).cpu().numpy()
    ref = oracle_mod.bruteforce(f, th, s, w)
    assert g_close(g64, ref) <= 1e-12
    assert g_close(g32, ref) <= 2e-5


def test_concurrent_host_pointer_calls_on_one_context(ctx, oracle_mod):
    # host-pointer calls stage through the context's buffer one at a time;
    # four threads calling at once each get their own image's result
    import threading
    imgs = [inputs(61 + 7 * i, 97 + 5 * i, 500 + i) for i in range(4)]
    refs = [oracle_mod.fabf(f, th, s, 4, 5)[0] for f, th, s in imgs]
    outs = [np.zeros(im[0].shape, np.float64) for im in imgs]
    errs = []

    def work(i):
        try:
            for _ in range(3):
                f, th, s = imgs[i]
                fabf.fabf_filter(ctx, f, th, s, 4, 5, out=outs[i])
        except Exception as e:   # noqa: BLE001 - reported below
            errs.append(e)

    ts = [threading.Thread(target=work, args=(i,)) for i in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errs
    for o, r in zip(outs, refs):
        assert g_close(o, r) <= RTOL_G


@pytest.mark.parametrize("H,W,w,N", [(65535, 3, 2, 5), (3, 65535, 2, 5), (65535, 70, 40, 6)])
def test_maximum_dimensions(ctx, oracle_mod, H, W, w, N):
    # the largest height / width the ABI accepts (65535), every pixel computed,
    # sampled pixels (and the four corners) checked against the oracle
    f, th, s = inputs(H, W, 900 + W, n_blobs=10)
    out = fabf.fabf_filter(ctx, dev(f), dev(th), dev(s), w, N)
    st, _ = fabf.fabf_get_status(ctx)
    assert st == fabf.FABF_OK
    g = out.cpu().numpy()
    rng = np.random.default_rng(H + W)
    ys = np.concatenate([rng.integers(0, H, 1500), [0, 0, H - 1, H - 1]])
    xs = np.concatenate([rng.integers(0, W, 1500), [0, W - 1, 0, W - 1]])
    ref, _ = oracle_mod.fabf_pixels(f, th, s, w, N, ys, xs)
    assert g_close(g[ys, xs], ref) <= RTOL_G
    assert np.isfinite(g).all()


def test_oversize_dimensions_rejected(ctx):
    f = torch.zeros((2, 65536), dtype=torch.uint8, device="cuda")
    th = torch.zeros((2, 65536), dtype=torch.float32, device="cuda")
    _, rc = fabf.fabf_filter(ctx, f, th, th, 2, 3, check=False)
    assert rc == fabf.FABF_EINVAL


@pytest.mark.parametrize("H,W,w,N,f64,pitch_extra", [(1080, 1920, 20, 5, False, 0), (96, 160, 5, 5, True, 0),
                                                     (17, 250, 3, 4, True, 5), (8, 64, 1, 2, False, 0),
                                                     (301, 77, 40, 6, True, 3)])
def test_pinned_host_buffers_equal_device_path(ctx, H, W, w, N, f64, pitch_extra):
    # pinned theta, sigma and out are read and written in place by the kernel
    # (only the image is copied); pinned or pageable image; the result must
    # equal the device-pointer call bit for bit, in every form
    f, th, s = inputs(H, W, 900 + H)
    pitch = W + pitch_extra
    buf = np.zeros((H, pitch), np.uint8)
    buf[:, :W] = f
    odt = torch.float64 if f64 else torch.float32
    pth, psg = torch.from_numpy(th).pin_memory(), torch.from_numpy(s).pin_memory()
    for prec in (fabf.FABF_FP64, fabf.FABF_CFP32, fabf.FABF_C32):
        if prec != fabf.FABF_FP64 and f64:
            continue
        fabf.fabf_set_precision(ctx, prec)
        try:
            d = fabf.fabf_filter(ctx, dev(buf), dev(th), dev(s), w, N, out_is_f64=f64, pitch=pitch).cpu().numpy()
            for img in (buf, torch.from_numpy(buf).pin_memory(), dev(buf)):
                pout = torch.full((H, W), -1.0, dtype=odt).pin_memory()
                fabf.fabf_filter(ctx, img, pth, psg, w, N, out=pout, out_is_f64=f64, pitch=pitch)
                torch.cuda.synchronize()
                assert np.array_equal(pout.numpy(), d), (prec, np.abs(pout.numpy() - d).max())
            # mixed: pinned maps with a pageable output take the staged paths
            hout = np.full((H, W), -1.0, np.float64 if f64 else np.float32)
            fabf.fabf_filter(ctx, buf, pth, psg, w, N, out=hout, out_is_f64=f64, pitch=pitch)
            assert np.array_equal(hout, d)
        finally:
            fabf.fabf_set_precision(ctx, fabf.FABF_FP64)


@pytest.mark.parametrize("H,W,w,N,f64,pitch_extra", [(1080, 1920, 20, 5, False, 0), (96, 160, 5, 5, True, 0),
                                                     (17, 250, 3, 4, True, 5), (8, 64, 1, 2, False, 0),
                                                     (301, 77, 40, 6, True, 3)])
def test_pipelined_host_path_equals_device_path(ctx, H, W, w, N, f64, pitch_extra):
    # host buffers go through the banded copy / compute / copy-back pipeline;
    # the result must equal the device-pointer call bit for bit, in every form
    f, th, s = inputs(H, W, 700 + H)
    pitch = W + pitch_extra
    buf = np.zeros((H, pitch), np.uint8)
    buf[:, :W] = f
    for prec in (fabf.FABF_FP64, fabf.FABF_CFP32, fabf.FABF_C32):
        if prec != fabf.FABF_FP64 and f64:
            continue
        fabf.fabf_set_precision(ctx, prec)
        try:
            host_out = np.zeros((H, W), np.float64 if f64 else np.float32)
            fabf.fabf_filter(ctx, buf, th, s, w, N, out=host_out, out_is_f64=f64, pitch=pitch)
            d = fabf.fabf_filter(ctx, dev(buf), dev(th), dev(s), w, N, out_is_f64=f64, pitch=pitch).cpu().numpy()
            torch.cuda.synchronize()
        finally:
            fabf.fabf_set_precision(ctx, fabf.FABF_FP64)
        assert np.array_equal(host_out, d), (prec, np.abs(host_out - d).max())


def test_pinned_host_buffers_report_status_and_clear_it(ctx):
    # the pinned-buffer path reads the kernels' status words from mapped host
    # memory: a non-positive sigma gives FABF_EINVAL (and NaN at that pixel),
    # and the next call starts from clear words
    f, th, s = inputs(70, 90, 5)
    pth = torch.from_numpy(th).pin_memory()
    bad = s.copy()
    bad[10, 11] = 0.0
    psg_bad = torch.from_numpy(bad).pin_memory()
    psg = torch.from_numpy(s).pin_memory()
    pout = torch.zeros((70, 90), dtype=torch.float64).pin_memory()
    img = torch.from_numpy(f).pin_memory()
    for prec in (fabf.FABF_FP64, fabf.FABF_C32):
        fabf.fabf_set_precision(ctx, prec)
        try:
            _, rc = fabf.fabf_filter(ctx, img, pth, psg_bad, 3, 5, out=pout, check=False)
            assert rc == fabf.FABF_EINVAL
            assert np.isnan(pout.numpy()[10, 11]) and np.isfinite(np.delete(pout.numpy().ravel(), 10 * 90 + 11)).all()
            _, rc = fabf.fabf_filter(ctx, img, pth, psg, 3, 5, out=pout, check=False)
            assert rc == fabf.FABF_OK
            st, _ = fabf.fabf_get_status(ctx)
            assert st == fabf.FABF_OK
        finally:
            fabf.fabf_set_precision(ctx, fabf.FABF_FP64)
