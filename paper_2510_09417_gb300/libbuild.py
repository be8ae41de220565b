"""Builds libvqhull.so (the CUDA kernels and the C ABI of include/vqhull.h)
in-tree with nvcc for sm_103a.  Translation units compile in parallel."""
from __future__ import annotations

import os
import platform
import subprocess
import sys
import threading
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build", platform.machine())
LIB = os.path.join(HERE, "libvqhull.so")
STAMP = os.path.join(BUILD, "lib.arch")
SOURCES = ["vq_kernels.cu", "vq_partition.cu", "vq_api.cu", "vq_server.cu", "vq_noalloc.cu"]
HEADERS = [os.path.join(CSRC, h) for h in ("vq_device.cuh", "vq_internal.h", "vq_common.cuh", "vq_partition.cuh",
                                            "vq_sieve.cuh", "vq_small.cuh", "vq_worklist.cuh", "vq_admit.h")] + [
    os.path.join(ROOT, "include", "vqhull.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]
# VQ_CHECKED=1 builds a library whose kernels validate computed indices
# (debugging aid; the default build has no checks)
CHECKED = os.environ.get("VQ_CHECKED", "") == "1"
if CHECKED:
    FLAGS = FLAGS + ["-DVQ_CHECKED=1"]
# VQ_K1_PROFILE=1 adds per-phase cycle counters to the partition kernel,
# printed to stderr after each call (profiling aid; off by default)
if os.environ.get("VQ_K1_PROFILE", "") == "1":
    FLAGS = FLAGS + ["-DVQ_K1_PROFILE=1"]
# VQ_WL_PROFILE=1 adds task counts and time sums to the persistent worklist,
# printed to stderr after each call (profiling aid; off by default)
if os.environ.get("VQ_WL_PROFILE", "") == "1":
    FLAGS = FLAGS + ["-DVQ_WL_PROFILE=1"]
_lock = threading.Lock()


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the library if any source or header is newer than it."""
    with _lock:
        srcs = [os.path.join(CSRC, s) for s in SOURCES]
        # a library built on another machine type (e.g. copied to an Arm
        # host) is rebuilt
        tag = platform.machine() + "".join(f for f in (" -DVQ_CHECKED=1", " -DVQ_K1_PROFILE=1", " -DVQ_WL_PROFILE=1")
                                           if f.strip() in FLAGS)
        same_arch = os.path.exists(STAMP) and open(STAMP).read().strip() == tag
        if not force and same_arch and not _stale(LIB, srcs + HEADERS + [__file__]):
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        nvcc = _nvcc()

        def compile_one(src):
            obj = os.path.join(BUILD, os.path.basename(src) + ".o")
            if force or not same_arch or _stale(obj, [src] + HEADERS + [__file__]):
                cmd = [nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj + ".tmp"]
                if verbose:
                    print(" ".join(cmd), file=sys.stderr)
                subprocess.check_call(cmd)
                os.replace(obj + ".tmp", obj)
            return obj

        with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
            objs = list(ex.map(compile_one, srcs))
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"])
        os.replace(tmp, LIB)
        with open(STAMP, "w") as f:
            f.write(tag)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
