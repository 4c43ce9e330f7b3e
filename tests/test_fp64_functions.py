"""The FP64 integrals use the library's own binary64 erfcx and exp
(fabf_device.cuh: piecewise Chebyshev interpolants of erfcx, Tang's
table-driven exp).  A host build of the same code and tables (nvcc) is
checked here against mpmath at 40 digits: within 2 units in the last place
of the true value over the whole argument range the FP64 integrals use
(erfcx on [0, inf], exp on [-745, 709], the subnormal range included).  The
committed table header must be what its generator writes."""
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1811_02308_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("fp64") / "fp64_check")
    res = subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-ffp-contract=off",
                          "-o", exe, os.path.join(HERE, "fp64_functions_check.cu")], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-2000:]

    def run(kind, xs):
        inp = "".join("%s %s\n" % (kind, float(x).hex()) for x in xs)
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split()
        return [float.fromhex(v) for v in out]
    return run


def ulps(got, ref):
    """|got - ref| in units of the last place of the binary64 value nearest ref
    (for subnormal results, of the subnormal spacing)."""
    r = float(ref)
    if r == 0.0:
        return 0.0 if got == 0.0 else float("inf")
    spacing = float(np.spacing(np.float64(abs(r))))
    return float(abs(mp.mpf(got) - ref) / spacing)


def test_erfcx_within_two_ulps(checker):
    mp.mp.dps = 40
    rng = np.random.default_rng(1)
    xs = list(rng.uniform(0, 8, 3000)) + list(np.exp(rng.uniform(np.log(8), np.log(1e6), 800)))
    xs += [i / 4 for i in range(33)] + [np.nextafter(i / 4, 0) for i in range(1, 33)]
    xs += [0.0, 1e-300, 5e-324, 1e-8, 7.999999999999999, 8.0, 1e10, 1e150, 1e300]
    got = checker("erfcx", xs)
    worst = 0.0
    for x, g in zip(xs, got):
        xm = mp.mpf(x)
        if x < 1e5:
            ref = mp.exp(xm * xm) * mp.erfc(xm)
        else:   # the asymptotic series, far inside its accuracy there
            u = 1 / (2 * xm * xm)
            ref = (1 - u + 3 * u * u - 15 * u ** 3) / (xm * mp.sqrt(mp.pi))
        worst = max(worst, ulps(g, ref))
    assert worst <= 2.0, worst
    assert checker("erfcx", [float("inf")]) == [0.0]


def test_exp_within_two_ulps(checker):
    mp.mp.dps = 40
    rng = np.random.default_rng(2)
    xs = list(rng.uniform(-745, 709, 3000)) + list(rng.uniform(-1, 1, 1000))
    xs += list(rng.uniform(-745.1, -708, 500))                      # subnormal results
    xs += [0.0, -0.0, 1e-300, -1e-17, 1e-17, -0.5, -1.0, -708.3964185322641, -709.0, -744.4400719213812, 709.0]
    got = checker("exp", xs)
    worst = 0.0
    for x, g in zip(xs, got):
        ref = mp.exp(mp.mpf(x))
        worst = max(worst, ulps(g, ref))
    assert worst <= 2.0, worst
    assert checker("exp", [-745.3, -1000.0, -float("inf")]) == [0.0, 0.0, 0.0]


def test_table_header_is_the_generators_output():
    res = subprocess.run([sys.executable, os.path.join(CSRC, "gen_fp64_tables.py")], capture_output=True, text=True,
                         check=True)
    with open(os.path.join(CSRC, "fabf_fp64_tables.h")) as fh:
        assert fh.read() == res.stdout


def test_double_to_float_rounding_is_ieee(checker):
    """The FP64-fit form rounds its binary64 coefficients to binary32 from the
    bits (double_to_float_rn); the result equals IEEE round-to-nearest-even
    (numpy's cast) on random values over the whole binary32 range, on exact
    ties of both parities, at the range edges and past them."""
    rng = np.random.default_rng(9)
    mant = rng.integers(0, 1 << 52, 4000, dtype=np.uint64)
    expo = rng.integers(1023 - 160, 1023 + 140, 4000, dtype=np.uint64)
    sign = rng.integers(0, 2, 4000, dtype=np.uint64) << np.uint64(63)
    xs = list((sign | (expo << np.uint64(52)) | mant).view(np.float64))
    # ties: the 29 discarded bits exactly one half, with even and odd kept bits
    for k in range(200):
        kept = int(rng.integers(0, 1 << 23))
        e = int(rng.integers(1023 - 126, 1023 + 128))
        xs.append(np.uint64((e << 52) | (kept << 29) | (1 << 28)).view(np.float64).item())
    big = float(np.finfo(np.float32).max)
    xs += [0.0, -0.0, 1.0, -1.0, big, np.nextafter(big, np.inf), big * (1 + 2.0 ** -25), big * (1 + 2.0 ** -24),
           float(np.finfo(np.float32).tiny), 1e-39, -1e-45, 1e-50, 1e300, -1e300, float("inf"), 3.4028235677973366e38]
    got = np.array(checker("d2f", xs))
    with np.errstate(over="ignore"):
        ref = np.array(xs, dtype=np.float64).astype(np.float32).astype(np.float64)
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
