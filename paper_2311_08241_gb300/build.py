"""Build libsesw.so in-tree with nvcc for sm_103a (GB300).

The translation units compile in parallel; the shared library links the CUDA
runtime statically so it does not depend on a runtime library path.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libsesw.so")
SOURCES = ["sesw_kernels.cu", "sesw_persistent.cu", "sesw_persistent_sesm.cu", "sesw_persistent_stream.cu",
           "sesw_persistent_sesm_stream.cu", "sesw_tc.cu", "sesw_noalloc.cu", "sesw_surrogate.cu",
           "sesw_api.cpp", "mesh_prep.cpp"]
HEADERS = [os.path.join(CSRC, "sesw_internal.h"), os.path.join(CSRC, "sesw_device.cuh"), os.path.join(CSRC, "sesw_msg.cuh"),
           os.path.join(CSRC, "sesw_persistent.cuh"),
           os.path.join(ROOT, "include", "sesw.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsesw")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, extra):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    deps = [os.path.join(CSRC, src)] + HEADERS
    if not _stale(obj, deps):
        return obj
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
           "-I", os.path.join(ROOT, "include"), *extra, "-c", os.path.join(CSRC, src), "-o", obj + ".tmp"]
    subprocess.run(cmd, check=True)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, extra=()) -> str:
    """Compile (when sources changed) and return the path of libsesw.so."""
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for f in os.listdir(BUILD):
            os.remove(os.path.join(BUILD, f))
    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, list(extra)), SOURCES))
    if _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run([nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs], check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
