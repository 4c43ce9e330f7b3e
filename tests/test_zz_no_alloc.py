"""fabf_filter_noalloc, the entry point for callers that cannot allocate
device memory (a real-time thread that cannot absorb cudaMalloc's
device-wide synchronisation, a plugin whose host framework owns every
allocation).  It keeps the kernel's status word and fallback counter in an
array compiled into the library instead of a context's cudaMalloc'd words.

Checked through the C ABI against the context-based fabf_filter on two
consecutive calls (bit for bit: the same FP64 kernel runs), so that the
second call shows the shared scratch was cleared, and against the CPU
oracle.  This file is collected last; it also passes alone in a fresh
process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1811_02308_gb300 import build, fabf, synth  # noqa: E402

pytestmark = pytest.mark.gpu

RTOL_G = 1e-9     # the output tolerance of the parity tests against the oracle


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1.0)))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    c = fabf.Context(device=0)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _pitched(f, pitch):
    """The image in a device buffer whose rows are `pitch` bytes apart."""
    H, W = f.shape
    buf = np.zeros((H, pitch), np.uint8)
    buf[:, :W] = f
    return _dev(buf)


CASES = [
    # H, W, w, N, seed, sigma range, zeta range, pitch (None: W), float64 output
    (256, 256, 5, 5, 11, (10, 40), None, None, True),
    (301, 517, 20, 6, 12, (5, 60), (-20, 20), None, True),
    (181, 250, 9, 4, 14, (5, 60), (-20, 20), 272, True),    # pitch > W, 16-byte rows: TMA
    (97, 130, 7, 5, 15, (5, 60), (-20, 20), 131, False),    # odd pitch (plain load), float32 output
]


def test_noalloc_matches_fabf_filter_and_oracle_on_two_calls(ctx, oracle_mod):
    for H, W, w, N, seed, sig, zeta, pitch, f64 in CASES:
        f, th, s = synth.make_inputs(H, W, seed, n_blobs=20, sigma_range=sig, zeta_range=zeta)
        p = W if pitch is None else pitch
        df = _dev(f) if pitch is None else _pitched(f, p)
        dth, ds = _dev(th), _dev(s)
        odt = torch.float64 if f64 else torch.float32
        ref = torch.empty((H, W), dtype=odt, device="cuda")
        fabf.fabf_filter(ctx, df, dth, ds, w, N, out=ref, out_is_f64=f64, pitch=p)
        torch.cuda.synchronize()
        st_ref, nf_ref = fabf.fabf_get_status(ctx)
        g_ref, nf_oracle = oracle_mod.fabf(f, th, s, w, N)
        for _ in range(2):                     # two calls in a row share the scratch
            out = torch.full((H, W), float("nan"), dtype=odt, device="cuda")
            rc, nf = fabf.fabf_filter_noalloc(df, dth, ds, w, N, out, out_is_f64=f64, pitch=p)
            assert rc == fabf.FABF_OK == st_ref
            assert nf == nf_ref == nf_oracle   # the counter was cleared, not accumulated
            got = out.cpu().numpy()
            assert np.array_equal(got, ref.cpu().numpy()), (H, W, w, N)
            if f64:
                assert _rel(got, g_ref) <= RTOL_G
            else:
                # float32 output: the FP64 result rounded once to binary32
                assert _rel(got, g_ref) <= 2.0 ** -24 + RTOL_G


def test_noalloc_allocates_nothing(ctx):
    """After a warm-up call, neither torch's caching allocator nor the
    device's free memory changes across calls."""
    H, W = 200, 333
    f, th, s = synth.make_inputs(H, W, 16, n_blobs=20, sigma_range=(5, 60), zeta_range=(-20, 20))
    df, dth, ds = _dev(f), _dev(th), _dev(s)
    out = torch.empty((H, W), dtype=torch.float64, device="cuda")
    rc, _ = fabf.fabf_filter_noalloc(df, dth, ds, 8, 5, out)
    assert rc == fabf.FABF_OK
    torch.cuda.synchronize()
    reserved0 = torch.cuda.memory_reserved()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        rc, _ = fabf.fabf_filter_noalloc(df, dth, ds, 8, 5, out)
        assert rc == fabf.FABF_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_reserved() == reserved0
    assert free1 == free0


def test_noalloc_clears_status_between_calls_and_rejects_host_buffers(ctx):
    f, th, s = synth.make_inputs(40, 50, 13, n_blobs=4)
    bad = s.copy()
    bad[2, 3] = -1.0
    out = torch.empty((40, 50), dtype=torch.float64, device="cuda")
    rc, _ = fabf.fabf_filter_noalloc(_dev(f), _dev(th), _dev(bad), 3, 4, out)
    assert rc == fabf.FABF_EINVAL
    rc, _ = fabf.fabf_filter_noalloc(_dev(f), _dev(th), _dev(s), 3, 4, out)
    assert rc == fabf.FABF_OK
    ref = fabf.fabf_filter(ctx, _dev(f), _dev(th), _dev(s), 3, 4)
    assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy())
    host_out = np.empty((40, 50), np.float64)
    rc, _ = fabf.fabf_filter_noalloc(f, th, s, 3, 4, host_out)
    assert rc == fabf.FABF_EINVAL


def test_noalloc_rejects_buffers_of_another_gpu(ctx):
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    f, th, s = synth.make_inputs(40, 50, 13, n_blobs=4)
    out = torch.empty((40, 50), dtype=torch.float64, device="cuda:0")
    lib = fabf.load()
    import ctypes as C
    other = torch.from_numpy(th).to("cuda:1")
    nf = C.c_uint64(0)
    with torch.cuda.device(0):
        rc = lib.fabf_filter_noalloc(_dev(f).data_ptr(), other.data_ptr(), _dev(s).data_ptr(), 40, 50, 50, 3, 4,
                                     out.data_ptr(), 1, 0, C.byref(nf))
    assert rc == fabf.FABF_EINVAL
