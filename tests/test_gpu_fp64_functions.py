"""The FP64 form's own erfcx and exp on the GPU equal their host build bit for
bit (the same IEEE operations and fused multiply-adds on both sides), and
the host build is within 2 units in the last place of mpmath
(tests/test_fp64_functions.py).  The host program is built here with nvcc
from the same header."""
import os
import shutil
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1811_02308_gb300 import build, fabf  # noqa: E402

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    c = fabf.Context(device=0)
    yield c
    c.close()


def host_values(tmp_path, kind, xs):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "fp64_check")
    if not os.path.exists(exe):
        res = subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler",
                              "-ffp-contract=off", "-o", exe, os.path.join(HERE, "fp64_functions_check.cu")],
                             capture_output=True, text=True)
        assert res.returncode == 0, res.stderr[-2000:]
    inp = "".join("%s %s\n" % (kind, float(x).hex()) for x in xs)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split()
    return np.array([float.fromhex(v) for v in out])


def test_device_equals_host_build(ctx, tmp_path):
    rng = np.random.default_rng(7)
    xs = np.concatenate([rng.uniform(0, 8, 20000), np.exp(rng.uniform(np.log(8), np.log(1e6), 4000)),
                         rng.uniform(0, 745.1, 4000), np.arange(33) / 4.0, [0.0, 5e-324, 1e-300, 1e300]])
    e1, e2 = fabf.fabf_debug_fp64_functions(ctx, torch.from_numpy(xs).cuda())
    g1, g2 = e1.cpu().numpy(), e2.cpu().numpy()
    h1 = host_values(tmp_path, "erfcx", xs)
    h2 = host_values(tmp_path, "exp", -xs)
    assert np.array_equal(g1.view(np.uint64), h1.view(np.uint64))
    assert np.array_equal(g2.view(np.uint64), h2.view(np.uint64))
