"""Build liblbm.so (the CUDA library behind include/lbm.h) in the package
directory with nvcc for sm_103a.  Objects go to _build/ next to it."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "liblbm.so")
SOURCES = ["lbm_kernels.cu", "lbm_kernels_f16.cu", "lbm_kernels_bf16.cu", "lbm_kernels_16x8x4.cu",
           "lbm_kernels_16x4x8.cu", "lbm_kernels_32x4x4.cu", "lbm_capi.cpp", "lbm_noalloc.cu", "lbm_mlp.cu"]
HEADERS = [os.path.join(CSRC, "lbm_internal.h"), os.path.join(CSRC, "lbm_step.cuh"),
           os.path.join(ROOT, "include", "lbm.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _flags():
    return ["-std=c++20", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-O3",
            "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False, checked: bool = False) -> str:
    """Build liblbm.so; with checked=True build liblbm_checked.so instead, whose
    step kernels test every slot and cell index before use and report the
    first failure through lbm_step's error (a debugging aid)."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    objs, jobs = [], []
    suffix = "_checked" if checked else ""
    lib = LIB.replace(".so", suffix + ".so")
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + suffix + ".o")
        objs.append(o)
        if force or _stale(o, [s, *HEADERS]):
            extra = ["-x", "cu"] if src.endswith(".cu") else []
            defs = ["-DLBM_CHECKED"] if checked else []
            jobs.append([nvcc, *_flags(), *defs, *extra, "-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r

    with ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        list(ex.map(run, jobs))
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
