"""Colour images on the GPU (Sec. IV-C: channel by channel, width maps on
the luma) against the oracle: the luma bit for bit, the per-channel filter
within the FP64 bar, and the colour texture pipeline (whose passes quantise
their outputs, so a pixel within 1e-13 of a .5 boundary may round the other
way) within the bar on >= 99.9 % of the samples."""
import ctypes
import math

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


def rel(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)


def texture_cfg(w=4, N=5, k=2, sw=None, sN=None):
    sh = fabf.SharpenCfg(sw or w, N if sN is None else sN, 1.0, 10.0, 10.0, 40.0)
    return fabf.TextureCfg(w, N, k, 1.0, 8.0, 5.0, 60.0, 0.8, sh)


def lq(rho, sat):
    taps = synth.gaussian_taps(rho)
    return taps, int(math.floor(sat * float(int(taps.sum())) ** 2 + 0.5))


@pytest.mark.parametrize("H,W", [(67, 131), (1, 45), (33, 1), (256, 300)])
def test_luma_bit_exact(ctx, oracle_mod, H, W):
    rgb = synth.make_rgb(H, W, 3 + H, n_blobs=10)
    Y = fabf.fabf_luma(ctx, dev(rgb)).cpu().numpy()
    assert np.array_equal(Y, oracle_mod.luma(rgb))


@pytest.mark.parametrize("H,W,w,N,with_theta", [(70, 133, 5, 5, False), (70, 133, 5, 5, True),
                                                (1, 90, 3, 4, False), (45, 2, 2, 6, True)])
def test_filter_rgb_matches_oracle(ctx, oracle_mod, H, W, w, N, with_theta):
    rgb = synth.make_rgb(H, W, 50 + H, n_blobs=12)
    rng = np.random.default_rng(H + W)
    sigma = synth.smooth_field(H, W, 5.0, 60.0, rng)
    theta = None
    if with_theta:
        zeta = np.stack([synth.smooth_field(H, W, -20.0, 20.0, rng) for _ in range(3)], axis=-1)
        theta = (rgb.astype(np.float32) + zeta).astype(np.float32)
    g = fabf.fabf_filter_rgb(ctx, dev(rgb), None if theta is None else dev(theta), dev(sigma), w, N).cpu().numpy()
    st, _ = fabf.fabf_get_status(ctx)
    assert st == fabf.FABF_OK
    ref = oracle_mod.filter_rgb(rgb, theta, sigma, w, N)
    assert rel(g, ref).max() <= RTOL_G


def test_filter_rgb_binary32_output(ctx, oracle_mod):
    # float32 output: the FP64 result rounded once
    rgb = synth.make_rgb(40, 57, 9, n_blobs=8)
    sigma = synth.smooth_field(40, 57, 5.0, 60.0, np.random.default_rng(2))
    g = fabf.fabf_filter_rgb(ctx, dev(rgb), None, dev(sigma), 4, 5, out_is_f64=False).cpu().numpy()
    ref = oracle_mod.filter_rgb(rgb, None, sigma, 4, 5)
    assert np.abs(g.astype(np.float64) - ref).max() <= 255 * 2.0 ** -24 + 1e-9


@pytest.mark.parametrize("H,W,sw,sN", [(80, 144, None, None), (37, 61, 2, 6), (1, 45, None, None), (29, 1, 3, 4)])
def test_texture_rgb_matches_oracle(ctx, oracle_mod, H, W, sw, sN):
    rgb = synth.make_rgb(H, W, 31 + W, n_blobs=15)
    g = fabf.fabf_texture_filter_rgb(ctx, dev(rgb), texture_cfg(sw=sw, sN=sN)).cpu().numpy()
    st, _ = fabf.fabf_get_status(ctx)
    assert st == fabf.FABF_OK
    taps, Lq = lq(1.0, 10.0)
    ref = oracle_mod.texture_filter_rgb(rgb, 4, 5, 2, 1.0, 8.0, 5.0, 60.0, taps, Lq, 10.0, 40.0, sw=sw, sN=sN)
    ok = rel(g, ref) <= RTOL_G
    assert ok.mean() >= 0.999, ok.mean()


def test_texture_rgb_on_replicated_gray_equals_gray_pipeline(ctx):
    f, _, _ = synth.make_inputs(64, 96, 77, n_blobs=12)
    rgb = np.ascontiguousarray(np.stack([f, f, f], axis=-1))
    cfg = texture_cfg()
    g3 = fabf.fabf_texture_filter_rgb(ctx, dev(rgb), cfg).cpu().numpy()
    g1 = fabf.fabf_texture_filter(ctx, dev(f), cfg).cpu().numpy()
    for c in range(3):
        assert np.array_equal(g3[..., c], g1)


def test_texture_rgb_binary32_form(ctx):
    rgb = synth.make_rgb(96, 160, 41, n_blobs=20)
    d = dev(rgb)
    g64 = fabf.fabf_texture_filter_rgb(ctx, d, texture_cfg()).cpu().numpy()
    fabf.fabf_set_precision(ctx, fabf.FABF_CFP32)
    try:
        g32 = fabf.fabf_texture_filter_rgb(ctx, d, texture_cfg(), out_is_f64=False).cpu().numpy()
    finally:
        fabf.fabf_set_precision(ctx, fabf.FABF_FP64)
    err = np.abs(g32.astype(np.float64) - g64)
    # intermediate roundings may flip a pixel by one gray level and spread.
    # Where the FP64 output leaves [0, 255] the sharpening centre lies in a
    # gap of the window's histogram under a narrow kernel: T2 is near zero and
    # the output moves by tens of gray levels when one input sample moves by
    # one level (seen: 809 against 937 for one sample 196 against 197).  Such
    # samples are rare and are left out of the RMS.
    inside = (g64 >= 0.0) & (g64 <= 255.0)
    assert inside.mean() >= 0.999
    assert np.sqrt(np.mean(err[inside] ** 2)) <= 0.1 and np.mean(err <= 0.5) >= 0.99


@pytest.mark.parametrize("prec", [0, 2])
def test_texture_rgb_is_the_composition_of_public_calls(ctx, prec):
    # the pipeline equals, bit for bit, the same steps taken through the
    # public calls (luma, width maps, single-channel filter), in both forms
    rgb = synth.make_rgb(48, 72, 5, n_blobs=10)
    d = dev(rgb)
    cfg = texture_cfg()
    f64 = prec == 0

    def rnd(g):
        return dev(np.clip(np.rint(g.cpu().numpy()), 0, 255).astype(np.uint8))

    fabf.fabf_set_precision(ctx, prec)
    try:
        full = fabf.fabf_texture_filter_rgb(ctx, d, cfg, out_is_f64=f64).cpu().numpy()
        s1 = fabf.fabf_texture_sigma(ctx, fabf.fabf_luma(ctx, d), cfg)
        s2 = s1 * 0.8
        f3 = []
        for c in range(3):
            fc = d[..., c].contiguous()
            f2 = rnd(fabf.fabf_filter(ctx, fc, fc.float(), s1, 4, 5, out_is_f64=f64))
            f3.append(rnd(fabf.fabf_filter(ctx, f2, f2.float(), s2, 4, 5, out_is_f64=f64)))
        _, s3 = fabf.fabf_sharpen_maps(ctx, fabf.fabf_luma(ctx, torch.stack(f3, -1).contiguous()), cfg.sharpen)
        for c in range(3):
            th, _ = fabf.fabf_sharpen_maps(ctx, f3[c], cfg.sharpen)
            g = fabf.fabf_filter(ctx, f3[c], th, s3, 4, 5, out_is_f64=f64).cpu().numpy()
            assert np.array_equal(g, full[..., c])
    finally:
        fabf.fabf_set_precision(ctx, fabf.FABF_FP64)


def test_rgb_reject_bad_arguments(ctx):
    rgb = dev(synth.make_rgb(20, 20, 1, n_blobs=2))
    sg = torch.full((20, 20), 20.0, dtype=torch.float32, device="cuda")
    out = torch.empty((20, 20, 3), dtype=torch.float64, device="cuda")
    lib = fabf.load()
    h = ctx.handle
    # pitch below 3 W
    assert lib.fabf_filter_rgb(h, rgb.data_ptr(), None, sg.data_ptr(), 20, 20, 59, 3, 5, out.data_ptr(), 1,
                               0) == fabf.FABF_EINVAL
    # host output
    host = np.zeros((20, 20, 3), np.float64)
    assert lib.fabf_filter_rgb(h, rgb.data_ptr(), None, sg.data_ptr(), 20, 20, 60, 3, 5, host.ctypes.data, 1,
                               0) == fabf.FABF_EINVAL
    # w and N out of range
    assert lib.fabf_filter_rgb(h, rgb.data_ptr(), None, sg.data_ptr(), 20, 20, 60, 41, 5, out.data_ptr(), 1,
                               0) == fabf.FABF_EUNSUPPORTED
    assert lib.fabf_filter_rgb(h, rgb.data_ptr(), None, sg.data_ptr(), 20, 20, 60, 3, -1, out.data_ptr(), 1,
                               0) == fabf.FABF_EINVAL
    bad = texture_cfg(k=0)
    assert lib.fabf_texture_filter_rgb(h, rgb.data_ptr(), 20, 20, 60, ctypes.byref(bad), out.data_ptr(), 1,
                                       0) == fabf.FABF_EINVAL
    Y = torch.empty((20, 20), dtype=torch.uint8, device="cuda")
    assert lib.fabf_luma(h, rgb.data_ptr(), 20, 20, 60, Y.data_ptr(), 19, 0) == fabf.FABF_EINVAL
    with pytest.raises(ValueError):
        fabf.fabf_filter_rgb(ctx, rgb[:, :, :2].contiguous(), None, sg, 3, 5)
