"""Build libfdtd.so in-tree with nvcc for sm_103a.

Each .cu translation unit is compiled in parallel, then linked into one shared
library (static CUDA runtime, so the library loads without a GPU driver and
uses the caller's CUDA context and streams).  Artefacts go to _build/ next to
this file; a rebuild happens only when a source or header is newer.

A second variant, built beside it in _build_check/ with -DFDTD_CHECK=1, checks every global store
and TMA x origin of the fused kernels before it happens (a failing check is skipped and reported as
a device status): the stand-in for a memory checker.  FDTD_CHECK=1 in the environment makes the
binding load that variant.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
CHECK = os.environ.get("FDTD_CHECK", "") == "1"


def build_dir(check: bool = CHECK) -> str:
    return os.path.join(HERE, "_build_check" if check else "_build")


BUILD = build_dir()
LIB = os.path.join(BUILD, "libfdtd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(ROOT, "include", "fdtd.h"), os.path.abspath(__file__)]


def up_to_date(check: bool = CHECK) -> bool:
    lib = os.path.join(build_dir(check), "libfdtd.so")
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          check: bool = CHECK) -> str:
    bdir = build_dir(check)
    lib = os.path.join(bdir, "libfdtd.so")
    if not force and up_to_date(check):
        return lib
    os.makedirs(bdir, exist_ok=True)
    nv = nvcc()
    extra = (extra or []) + (["-DFDTD_CHECK=1"] if check else [])

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nv, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    srcs = _sources()
    with ThreadPoolExecutor(max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nv, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    v = "-v" in sys.argv
    xs = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=True, verbose=v, extra=xs))
