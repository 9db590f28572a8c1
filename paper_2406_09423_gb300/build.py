"""Builds libmsz.so (the CUDA library behind include/msz.h) in-tree.

Every .cu under csrc/ is compiled for sm_103a in parallel and linked into
paper_2406_09423_gb300/_build/libmsz.so, and a second time with MSZ_CHECKED
(bounds checks of every index read from device data, recording an error
instead of accessing) into libmsz_checked.so. Device code is compiled
without FMA contraction (-fmad=false) and host code with -ffp-contract=off,
so every floating-point step of the edit arithmetic is one IEEE
round-to-nearest operation.
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
LIB = os.path.join(OUT, "libmsz.so")
LIB_CHECKED = os.path.join(OUT, "libmsz_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the MSz CUDA library cannot be built")
    return cand


def _flags(extra=()):
    return ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-fmad=false",
            "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
            "-I", os.path.join(ROOT, "include"), "-I", CSRC, *extra]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(LIB_CHECKED)):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_CHECKED))
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "msz.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Builds both libraries (in parallel); returns the normal one's path."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()
    variants = {LIB: (), LIB_CHECKED: ("-DMSZ_CHECKED",)}

    def compile_one(job):
        src, lib, defs = job
        tag = "_checked" if defs else ""
        obj = os.path.join(OUT, os.path.basename(src)[:-3] + tag + ".o")
        cmd = [cc, *_flags(tuple(extra) + defs), "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, flush=True)
        return lib, obj

    jobs = [(src, lib, defs) for lib, defs in variants.items() for src in sources()]
    with ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        done = list(ex.map(compile_one, jobs))
    for lib in variants:
        objs = [o for l, o in done if l == lib]
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys

    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
    print(LIB)
