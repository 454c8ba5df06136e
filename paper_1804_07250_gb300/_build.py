"""Build libtiling.so in-tree with nvcc for sm_103a.

Each translation unit is compiled to an object in parallel, then linked into
one shared library next to this file.  Nothing is installed anywhere else.
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
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtiling.so")
# the bounds-checked build (-DTL_DEBUG): the binding loads it when TL_DEBUG=1
LIB_DEBUG = os.path.join(HERE, "libtiling_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["tl_kernels.cu", "tl_resident.cu", "tl_regdom.cu", "tl_batch.cu", "tl_shuffle.cu", "tl_host.cpp", "tl_thurston.cpp"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libtiling.so")
    return cand


def _compile(src: str, extra: list[str], build_dir: str = BUILD) -> str:
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-I", INCLUDE, "-I", CSRC,
           "-Xcompiler", "-fPIC,-fvisibility=hidden", "-Xptxas", "-warn-spills",
           "-c", os.path.join(CSRC, src), "-o", obj, *extra]
    subprocess.run(cmd, check=True)
    return obj


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "tiling.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False, debug: bool = False) -> str:
    """Build libtiling.so, or with `debug` the bounds-checked
    libtiling_debug.so (-DTL_DEBUG, objects in _build/debug)."""
    lib = LIB_DEBUG if debug else LIB
    bdir = os.path.join(BUILD, "debug") if debug else BUILD
    if not force and not _stale(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    if debug:
        extra += ["-DTL_DEBUG"]
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, bdir), srcs))
    tmp = lib + ".tmp.%d" % os.getpid()
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc())), "lib64")
    subprocess.run([nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
                    "-Xlinker", "-rpath," + cuda_lib], check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, debug="--debug" in sys.argv))
