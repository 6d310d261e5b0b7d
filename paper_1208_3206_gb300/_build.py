"""Build liblt.so (the sm_103a CUDA library behind include/lt.h) in-tree.

Each .cu file compiles in parallel into an object, then nvcc links the
shared library. Only one architecture is built: sm_103a (GB300).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblt.so")
SOURCES = ["lt_api.cu", "lt_build.cu", "lt_bin.cu", "lt_tile.cu", "lt_raster.cu", "lt_backward.cu", "lt_static.cu",
           "lt_resample.cu", "lt_slice.cu", "lt_centroids.cu", "lt_area.cu"]
HEADERS = ["lt_common.cuh", "lt_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(cuda, "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


STAMP = os.path.join(OUT_DIR, "flags.txt")  # the extra flags the library was built with


def _stale(extra) -> bool:
    if not os.path.exists(LIB):
        return True
    built_with = open(STAMP).read() if os.path.exists(STAMP) else None
    if built_with != " ".join(extra):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "lt.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    """Compile liblt.so if missing, older than its sources or built with
    other extra flags (a bounds-checking build, say); returns its path."""
    if not force and not _stale(list(extra_flags or [])):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    extra = list(extra_flags or [])

    def compile_one(src: str) -> str:
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as fh:
        fh.write(" ".join(extra))
    return LIB


if __name__ == "__main__":
    # --check-bounds: the debugging build whose index checks latch
    # LT_ERR_BOUNDS instead of touching memory out of range
    flags = (["-Xptxas", "-v"] if "--ptxas" in sys.argv else []) + \
        (["-DLT_CHECK_BOUNDS"] if "--check-bounds" in sys.argv else [])
    print(build(force="--force" in sys.argv or "--check-bounds" in sys.argv, verbose="-v" in sys.argv,
                extra_flags=flags or None))
