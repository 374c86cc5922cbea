"""Build libhelm.so (and the bounds-checking libhelm_debug.so) in-tree with nvcc
for sm_103a (no CMake, no torch extension).

Every translation unit of both libraries compiles in parallel; the shared
libraries are linked beside this file.  libhelm_debug.so is the same source
compiled with HELM_DEBUG: guard bands after every workspace array, host-side
slot-index checks, HELM_E_BOUNDS on a violation.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(HERE, "_build")
BUILD_DIR_DEBUG = os.path.join(HERE, "_build_debug")
LIB = os.path.join(HERE, "libhelm.so")
LIB_DEBUG = os.path.join(HERE, "libhelm_debug.so")

SOURCES = ["abi.cu", "solver.cu", "stencil.cu", "krylov.cu", "transfer.cu", "fwi.cu", "noalloc.cu", "batch.cu", "diag.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]
VARIANTS = {"release": (BUILD_DIR, LIB, []), "debug": (BUILD_DIR_DEBUG, LIB_DEBUG, ["-DHELM_DEBUG"])}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    deps.append(os.path.join(INCLUDE, "helm.h"))
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False, extra_flags=None, variants=("release", "debug")) -> str:
    cc = nvcc()
    extra = list(extra_flags or [])
    jobs, links = [], []
    for v in variants:
        bdir, lib, vflags = VARIANTS[v]
        os.makedirs(bdir, exist_ok=True)
        objs = []
        stale = False
        for s in SOURCES:
            src = os.path.join(CSRC, s)
            obj = os.path.join(bdir, s.replace(".cu", ".o"))
            objs.append(obj)
            if force or _stale(obj, src):
                jobs.append([cc, *ARCH, *FLAGS, *vflags, *extra, "-c", src, "-o", obj])
                stale = True
        if stale or not os.path.exists(lib):
            links.append([cc, *ARCH, "-shared", "-o", lib, *objs, "-lcudart"])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {cmd[-3]}")
        return r

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(run, jobs))
    for cmd in links:
        run(cmd)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
