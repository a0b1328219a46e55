"""Compile the CUDA library in-tree for sm_103a (nvcc, one -gencode).

Each translation unit is compiled in parallel into ``_build/obj`` and linked
into ``_build/libopal_gb300.so``.  Nothing is installed outside the package.
``build(timeline=True)`` makes the measurement build with the device
timeline (``OPAL_TIMELINE``) in ``_build_timeline/`` instead; the normal
library is never replaced by it.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libopal_gb300.so")
BUILD_TIMELINE = os.path.join(HERE, "_build_timeline")
LIB_TIMELINE = os.path.join(BUILD_TIMELINE, "libopal_gb300.so")
SOURCES = ["k_body.cu", "k_kick.cu", "k_scan.cu", "k_bs.cu", "k_bs_huge.cu", "k_energy.cu", "k_peaks.cu", "opal_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-diag-suppress", "1444"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is needed to build the library")


def _deps():
    return ([os.path.join(CSRC, s) for s in SOURCES] + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(ROOT, "include", "*.h")))


def up_to_date(timeline: bool = False) -> bool:
    lib = LIB_TIMELINE if timeline else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), timeline: bool = False) -> str:
    out_dir, lib = (BUILD_TIMELINE, LIB_TIMELINE) if timeline else (BUILD, LIB)
    if timeline:
        extra_flags = ("-DOPAL_TIMELINE", *extra_flags)
    elif extra_flags:
        raise ValueError("extra flags only with timeline=True: the normal library is built one way")
    if not force and up_to_date(timeline):
        return lib
    obj_dir = os.path.join(out_dir, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        out = os.path.join(obj_dir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", out]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr.strip():
            print(r.stderr)
        return out

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".{os.getpid()}.tmp"
    # --no-undefined: a symbol missing from every translation unit fails here, not at load time
    cmd = [cc, *ARCH, "-shared", "-Xlinker", "--no-undefined", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
