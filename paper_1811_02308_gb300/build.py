"""Build ``libfabf.so`` (the CUDA kernels plus the C ABI of include/fabf.h)
in-tree with nvcc for sm_103a.  Translation units compile in parallel."""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfabf.so")

SOURCES = [
    "fabf_inst_fp64.cu",
    "fabf_inst_fp64fit.cu",
    "fabf_inst_cfp32.cu",
    "fabf_inst_c32.cu",
    "fabf_inst_c32w.cu",
    "fabf_api.cu",
    "fabf_batch_serve.cu",
    "fabf_noalloc.cu",
    "fabf_sep.cu",
    "fabf_sep_p0.cu",
    "fabf_sep_p1.cu",
    "fabf_sep_p2.cu",
    "fabf_sep_p3.cu",
    "fabf_casc_p0.cu",
    "fabf_casc_p1.cu",
    "fabf_casc_p2.cu",
    "fabf_casc_p3.cu",
    "fabf_apps.cu",
    "fabf_peaks.cu",
]
HEADERS = ["fabf_device.cuh", "fabf_kernels.cuh", "fabf_launch.cuh", "fabf_internal.h", "fabf_sep_kernels.cuh",
           "fabf_casc_kernels.cuh", "fabf_fp64_tables.h"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfabf.so")


def _deps_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    paths.append(os.path.join(ROOT, "include", "fabf.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit and link ``libfabf.so``; return its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s" % (src, res.stderr[-4000:]))
        if verbose and res.stderr:
            print(res.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc link failed:\n%s" % res.stderr[-4000:])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
