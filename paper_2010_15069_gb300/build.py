"""Build the CUDA library libspgpe.so in-tree for sm_103a (GB300).

Each translation unit under csrc/ is compiled by nvcc in parallel into
_build/, then linked with cuFFT (used only by the comparator entry point).
Objects newer than their source and every header are reused.

build(bounds=True) builds the bounds-checked variant libspgpe_bounds.so into
_build_bounds/ (-DSPGPE_BOUNDS: every checked index outside its buffer sets an
error bit, reported as SPGPE_EBOUNDS, and the access is skipped), the
stand-in for a memory checker; processes select it with SPGPE_LIBRARY.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libspgpe.so")
OUT_BOUNDS = os.path.join(HERE, "_build_bounds")
LIB_BOUNDS = os.path.join(OUT_BOUNDS, "libspgpe_bounds.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the spgpe CUDA library cannot be built")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))


def build(force: bool = False, verbose: bool = False, jobs: int | None = None, bounds: bool = False) -> str:
    out_dir, lib_path = (OUT_BOUNDS, LIB_BOUNDS) if bounds else (OUT, LIB)
    flags = FLAGS + (["-DSPGPE_BOUNDS"] if bounds else [])
    os.makedirs(out_dir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    newest_hdr = max(os.path.getmtime(h) for h in _headers())
    cc = nvcc()

    def obj_of(src):
        return os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")

    def compile_one(src):
        obj = obj_of(src)
        if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), newest_hdr):
            return obj
        tmp = obj + f".tmp{os.getpid()}"
        cmd = [cc, *flags, *ARCH, "-c", src, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr[-4000:]}")
        if verbose and r.stderr:
            print(r.stderr)
        os.replace(tmp, obj)
        return obj

    with ThreadPoolExecutor(max_workers=jobs or min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    if force or not os.path.exists(lib_path) or os.path.getmtime(lib_path) < max(os.path.getmtime(o) for o in objs):
        tmp = lib_path + f".tmp{os.getpid()}"
        cudalib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(cc))), "lib64")
        cmd = [cc, "-shared", *ARCH, "-o", tmp, *objs, "-L", cudalib, "-lcufft",
               "-Xlinker", "-rpath", "-Xlinker", cudalib]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
