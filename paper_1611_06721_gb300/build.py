"""Builds the sm_103a shared library ``_lib/libmqs.so`` from ``csrc/`` with nvcc.

Each translation unit is compiled in parallel, then linked with
``nvcc -shared``.  Only ``-gencode arch=compute_103a,code=sm_103a`` is
emitted: the library targets GB300 only.

``build(debug=True)`` makes the debug variant ``_lib_debug/libmqs.so``
(``-DMQS_DEBUG_CHECKS``: every index a kernel computes is range-checked, every
device buffer carries guard bytes); the binding loads it when ``MQS_DEBUG=1``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libmqs.so")
OUT_DEBUG = os.path.join(HERE, "_lib_debug")
UNITS = ["pcg.cu", "pcg_mixed.cu", "conductor.cu", "mrhs.cu", "api.cu", "noalloc.cu", "adjoint.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmqs.so")
    return exe


def _newer(target: str, deps) -> bool:
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(d) <= t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    out = OUT_DEBUG if debug else OUT
    lib = os.path.join(out, "libmqs.so")
    flags = FLAGS + (["-DMQS_DEBUG_CHECKS"] if debug else [])
    os.makedirs(out, exist_ok=True)
    headers = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "mqs.h"))
    objs, jobs = [], []
    for u in UNITS:
        src = os.path.join(SRC, u)
        obj = os.path.join(out, u.replace(".cu", ".o"))
        objs.append(obj)
        if force or not _newer(obj, [src] + headers):
            jobs.append([nvcc(), *ARCH, *flags, "-c", src, "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        for cmd, res in zip(jobs, ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs)):
            if verbose or res.returncode != 0:
                sys.stderr.write(res.stdout + res.stderr)
            if res.returncode != 0:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    if force or jobs or not _newer(lib, objs):
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", lib, *objs, "-ldl"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            sys.stderr.write(res.stdout + res.stderr)
            raise RuntimeError("link failed: " + " ".join(cmd))
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
