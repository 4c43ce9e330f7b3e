"""The applications of Sec. IV on the GPU against the oracle: the sharpening
and texture maps bit for bit, one sharpening pass within the FP64 bar, and
the three-pass texture pipeline (whose passes quantise their outputs, so a
pixel within 1e-13 of a .5 boundary may round the other way) within the bar
on >= 99.9 % of the pixels."""
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


def sharpen_cfg(w=5, N=5, rho=1.0, sat=10.0, lo=10.0, hi=40.0):
    return fabf.SharpenCfg(w, N, rho, sat, lo, hi)


def texture_cfg(w=5, N=5, k=2, sh=None):
    return fabf.TextureCfg(w, N, k, 1.0, 8.0, 5.0, 60.0, 0.8, sh or sharpen_cfg(w, N))


def lq(rho, sat):
    taps = synth.gaussian_taps(rho)
    return taps, int(math.floor(sat * float(int(taps.sum())) ** 2 + 0.5))


@pytest.mark.parametrize("H,W,w,rho", [(67, 131, 5, 1.0), (1, 40, 3, 0.7), (50, 1, 2, 2.0), (130, 97, 40, 1.5)])
def test_sharpen_maps_bit_exact(ctx, oracle_mod, H, W, w, rho):
    f, _, _ = synth.make_inputs(H, W, 7 + H, n_blobs=20)
    cfg = sharpen_cfg(w=w, rho=rho, sat=12.0)
    th, sg = fabf.fabf_sharpen_maps(ctx, dev(f), cfg)
    torch.cuda.synchronize()
    taps, Lq = lq(rho, 12.0)
    assert np.array_equal(th.cpu().numpy(), oracle_mod.sharpen_theta(f, w))
    assert np.array_equal(sg.cpu().numpy(), oracle_mod.sharpen_sigma(f, taps, Lq, 10.0, 40.0))


@pytest.mark.parametrize("H,W,k", [(67, 131, 2), (1, 40, 1), (50, 1, 3), (90, 77, 6)])
def test_texture_sigma_bit_exact(ctx, oracle_mod, H, W, k):
    f, _, _ = synth.make_inputs(H, W, 11 + H, n_blobs=20)
    sg = fabf.fabf_texture_sigma(ctx, dev(f), texture_cfg(k=k))
    torch.cuda.synchronize()
    assert np.array_equal(sg.cpu().numpy(), oracle_mod.texture_sigma(f, k, 1.0, 8.0, 5.0, 60.0))


def test_sharpen_pass_matches_oracle(ctx, oracle_mod):
    f, _, _ = synth.make_inputs(96, 160, 21, n_blobs=20)
    cfg = sharpen_cfg(w=4, N=5)
    g = fabf.fabf_sharpen(ctx, dev(f), cfg).cpu().numpy()
    st, _ = fabf.fabf_get_status(ctx)
    assert st == fabf.FABF_OK
    taps, Lq = lq(1.0, 10.0)
    ref = oracle_mod.sharpen(f, 4, 5, taps, Lq, 10.0, 40.0)
    assert rel(g, ref).max() <= RTOL_G


@pytest.mark.parametrize("H,W", [(80, 144), (1, 57), (41, 1)])
def test_texture_pipeline_matches_oracle(ctx, oracle_mod, H, W):
    f, _, _ = synth.make_inputs(H, W, 31, n_blobs=20)
    g = fabf.fabf_texture_filter(ctx, dev(f), texture_cfg(w=4, N=5)).cpu().numpy()
    st, _ = fabf.fabf_get_status(ctx)
    assert st == fabf.FABF_OK
    taps, Lq = lq(1.0, 10.0)
    ref, _ = oracle_mod.texture_filter(f, 4, 5, 2, 1.0, 8.0, 5.0, 60.0, taps, Lq, 10.0, 40.0)
    ok = rel(g, ref) <= RTOL_G
    assert ok.mean() >= 0.999, ok.mean()


def test_texture_pipeline_binary32_form(ctx):
    # the pipeline in the compensated binary32 form against its FP64 form
    f, _, _ = synth.make_inputs(120, 200, 41, n_blobs=30)
    d = dev(f)
    g64 = fabf.fabf_texture_filter(ctx, d, texture_cfg()).cpu().numpy()
    fabf.fabf_set_precision(ctx, fabf.FABF_CFP32)
    try:
        g32 = fabf.fabf_texture_filter(ctx, d, texture_cfg(), out_is_f64=False).cpu().numpy()
    finally:
        fabf.fabf_set_precision(ctx, fabf.FABF_FP64)
    err = np.abs(g32.astype(np.float64) - g64)
    # intermediate roundings may flip a pixel by one gray level and spread
    assert np.sqrt(np.mean(err ** 2)) <= 0.1 and np.mean(err <= 0.5) >= 0.99


def test_apps_reject_bad_arguments(ctx):
    f, _, _ = synth.make_inputs(20, 20, 1)
    d = dev(f)
    out = torch.empty((20, 20), dtype=torch.float64, device="cuda")
    lib = fabf.load()
    bad = sharpen_cfg(w=0)
    assert lib.fabf_sharpen(ctx.handle, d.data_ptr(), 20, 20, 20, C_byref(bad), out.data_ptr(), 1, 0) == fabf.FABF_EINVAL
    bad = sharpen_cfg(lo=50.0, hi=40.0)
    assert lib.fabf_sharpen(ctx.handle, d.data_ptr(), 20, 20, 20, C_byref(bad), out.data_ptr(), 1, 0) == fabf.FABF_EINVAL
    bad = sharpen_cfg(rho=14.0)
    assert lib.fabf_sharpen(ctx.handle, d.data_ptr(), 20, 20, 20, C_byref(bad), out.data_ptr(), 1, 0) == fabf.FABF_EUNSUPPORTED
    host = np.zeros((20, 20), np.float64)
    assert lib.fabf_sharpen(ctx.handle, d.data_ptr(), 20, 20, 20, C_byref(sharpen_cfg()), host.ctypes.data, 1,
                            0) == fabf.FABF_EINVAL


def C_byref(x):
    import ctypes
    return ctypes.byref(x)
