"""Compile the CUDA library in-tree: csrc/*.cu -> libsb.so (sm_103a).

Each translation unit is compiled with nvcc for
``-gencode arch=compute_103a,code=sm_103a`` (``-lineinfo`` for profiling),
in parallel, then linked with the shared CUDA runtime.  A rebuild happens
only when a source or header is newer than the library.  ``checks=True``
builds the bounds-checked variant, libsb_checks.so (``-DSB_CHECKS``: index
checks that record a failure and skip the access; see include/sb.h).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libsb.so")
LIB_CHECKS = os.path.join(HERE, "libsb_checks.so")
BUILD_DIR = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsb.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "sb.h")]


def needs_build(checks: bool = False) -> bool:
    lib = LIB_CHECKS if checks else LIB
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, checks: bool = False) -> str:
    lib = LIB_CHECKS if checks else LIB
    if not force and not needs_build(checks):
        build_peak()
        return lib
    nvcc = _nvcc()
    obj_dir = os.path.join(BUILD_DIR, "checks") if checks else BUILD_DIR
    os.makedirs(obj_dir, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v" if verbose else "-O3",
                    "-I", os.path.join(ROOT, "include")] + (["-DSB_CHECKS"] if checks else [])

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src).replace(".cu", ".o"))
        cmd = [nvcc] + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    build_peak(force)
    return lib


PEAK_SRC = os.path.join(HERE, "peak", "int_peak.cu")
PEAK_LIB = os.path.join(HERE, "peak", "libsb_peak.so")


def build_peak(force: bool = False) -> str:
    """The instruction-rate microbenchmark (peak/int_peak.cu -> peak/libsb_peak.so)."""
    if not force and os.path.exists(PEAK_LIB) and os.path.getmtime(PEAK_LIB) >= os.path.getmtime(PEAK_SRC):
        return PEAK_LIB
    tmp = PEAK_LIB + ".tmp%d" % os.getpid()
    cmd = [_nvcc()] + ARCH + ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared",
                              PEAK_SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (PEAK_SRC, r.stdout, r.stderr))
    os.replace(tmp, PEAK_LIB)
    return PEAK_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checks="--checks" in sys.argv))
