"""The FP64 form divides the moments M_k and theta - alpha by powers d^k with
a correctly rounded reciprocal and one fused multiply-add correction
(div_by_power in fabf_device.cuh); the FP64 stage parity with the oracle
needs those quotients to be exactly IEEE's.  A host-only program built with
nvcc from the same header checks the reciprocal table and the correction
against IEEE division on every divisor d^k (d = 1..255, k = 1..6), for the
moments' range, for theta - alpha (t0, any sign) and for the separable
path's larger moments."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_division_by_powers_is_ieee_division(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "div_check")
    res = subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-ffp-contract=off",
                          "-o", exe, os.path.join(HERE, "div_by_power_check.cu")], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-2000:]
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    total, bad, bad_table, total2, bad2 = (int(v) for v in out)
    assert total == 255 * 6 * 2000 and total2 == 255 * 6 * 1000
    assert bad_table == 0
    assert bad == 0
    assert bad2 == 0
