"""Builds libofsc.so in-tree for sm_103a with nvcc (no cmake; translation units in parallel)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libofsc.so")
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
LIB_DEBUG = os.path.join(PKG, "libofsc_debug.so")
SOURCES = ["api.cu", "graph.cu", "iterate.cu", "spmm_dir.cu", "cluster.cu", "gram_tc.cu", "spmm_tma.cu", "direction_tc.cu", "ritz.cu", "wgrad.cu", "unroll.cu", "group.cu", "linesearch.cu"]
HEADERS = [os.path.join(CSRC, "common.cuh"), os.path.join(CSRC, "spmm_dir.cuh"), os.path.join(CSRC, "tcgen05.cuh"), os.path.join(CSRC, "cubic.cuh"), os.path.join(CSRC, "group.cuh"), os.path.join(CSRC, "spmm_dir_body.inc"), os.path.join(CSRC, "direction_body.inc"), os.path.join(ROOT, "include", "ofsc.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False, debug: bool = False) -> str:
    """Compiles every CUDA translation unit for sm_103a and links libofsc.so; returns its path.
    debug=True builds the checked library libofsc_debug.so instead (-DOFSC_DEBUG=1: the direction
    product checks its column indices and row ranges and the calls report a violation)."""
    bdir = BUILD_DEBUG if debug else BUILD
    lib = LIB_DEBUG if debug else LIB
    flags = FLAGS + (["-DOFSC_DEBUG=1"] if debug else [])
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + HEADERS):
            jobs.append([cc, *ARCH, *flags, "-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed ({' '.join(cmd)}):\n{r.stdout}\n{r.stderr}")
        return r

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        list(ex.map(run, jobs))
    if force or jobs or _stale(lib, objs):
        tmp = lib + ".tmp"
        run([cc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
