"""In-tree build of the CUDA library ``_build/libcvweno.so`` for sm_103a.

Every translation unit is compiled by nvcc in parallel (one -gencode, no cmake) and
linked into one shared library; the result is git-ignored and rebuilt when any
source or header is newer.

``build(checked=True)`` makes the bounds-checked variant ``_build/libcvweno_check.so``
(-DCVWENO_CHECK): the same entry points, with every global load and store of the stage
kernels checked against its array's extent; a failed check is reported as
CVWENO_ERR_CHECK by the next status check, and nothing traps.  The binding loads it
when CVWENO_CHECKED=1 is set in the environment.
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
LIB = os.path.join(BUILD, "libcvweno.so")
LIB_CHECK = os.path.join(BUILD, "libcvweno_check.so")
SOURCES = ["tables.cpp", "api.cu", "dg_scalar_1d.cu", "dg_scalar_2d.cu", "dg_euler.cu", "cg_scalar.cu", "noalloc.cu",
           "batch.cu", "dg_scalar_2d_mlp.cu", "surrogate.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcvweno.so")
    return exe


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    files.append(os.path.abspath(__file__))  # a change of the source list or flags
    return files


def lib_path(checked: bool = False) -> str:
    return LIB_CHECK if checked else LIB


def is_stale(checked: bool = False) -> bool:
    lib = lib_path(checked)
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False, jobs: int | None = None, checked: bool = False) -> str:
    lib = lib_path(checked)
    if not force and not is_stale(checked):
        return lib
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    pid = os.getpid()
    tag = "check." if checked else ""
    defs = ["-DCVWENO_CHECK"] if checked else []

    def compile_one(src):
        obj = os.path.join(BUILD, src + f".{tag}{pid}.o")
        cmd = [nvcc, *ARCH, *FLAGS, *defs, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=jobs or len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".{pid}.tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
