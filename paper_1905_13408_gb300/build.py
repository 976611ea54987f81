"""Build ``libspg.so`` (the C-ABI CUDA library) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library next to this file. No CMake, no Python extension module: the
binding loads the library with ctypes.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libspg.so")
# The checked build: every index of the fused step's shared-memory and global
# accesses is verified on the device (a failure records SPG_ECHECK and skips
# the access). Built on request only; used by the tests in place of a memory
# checker.
LIB_CHECK = os.path.join(HERE, "libspg_check.so")
SOURCES = ["spg_step_f32.cu", "spg_step_bf16.cu", "spg_step.cu", "spg_aux.cu", "spg_api.cu", "spg_noalloc.cu",
           "spg_fsc.cu", "spg_cufft.cu", "spg_fourier.cu", "spg_grid.cu", "spg_zfft.cu", "spg_xpass.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(verbose=False, checked=False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                "--expt-relaxed-constexpr"]
    if checked:
        f += ["-DSPG_CHECK"]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES]
    deps += [os.path.join(CSRC, "spg_internal.h"), os.path.join(CSRC, "spg_step_kernel.cuh"),
             os.path.join(CSRC, "spg_cufft.h"), os.path.join(CSRC, "spg_trace.h"), os.path.join(CSRC, "spg_fft.cuh"),
             os.path.join(INCLUDE, "spg.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, checked=False):
    """Compile and link; returns the library path (the checked build with
    checked=True)."""
    lib = LIB_CHECK if checked else LIB
    if not force and not _stale(lib):
        return lib
    cc = nvcc()
    objdir = os.path.join(HERE, "_build_check" if checked else "_build")
    os.makedirs(objdir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(verbose, checked)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stderr}")
        return obj, res.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, "-shared", "-o", tmp] + [o for o, _ in results] + ARCH + ["-Xcompiler", "-fPIC", "-ldl"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
