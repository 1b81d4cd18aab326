"""Compile the PEOs CUDA library (libpeos.so) in-tree for sm_103a with nvcc.

Every translation unit is compiled with --fmad=false (no contraction of a*b+c:
the routing-test and code-builder arithmetic is written in a fixed rounding
order) and host code with -ffp-contract=off.  Objects compile in parallel.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libpeos.so")
# the self-checked library (-DPEOS_CHECKED: index and list-invariant checks in the search
# kernel, counted instead of faulting; peos_check_read)
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(BUILD_CHECKED, "libpeos.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["api.cu", "search.cu", "search_bf16.cu", "search_e4m3.cu", "search_cw3_f32.cu", "search_cw3_bf16.cu",
           "search_cw3_e4m3.cu", "search_beam_f32.cu", "search_beam_bf16.cu", "search_beam_e4m3.cu", "build.cu",
           "knn.cu", "quant.cu", "noalloc.cu", "rng.cpp", "server.cpp", "knn_tc.cu", "perm.cu", "hier.cu",
           "simhash.cu", "index_io.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the PEOs library needs the CUDA toolkit to build")


def _flags():
    return ["-O3", "-std=c++17", *ARCH, "-lineinfo", "--fmad=false", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
            "-I", INCLUDE, "-I", CSRC]


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "peos.h"), __file__]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    out_dir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    if not force and not _stale(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    objs = []
    cmds = []
    extra = ["-DPEOS_CHECKED"] if checked else []
    for src in SOURCES:
        obj = os.path.join(out_dir, src + ".o")
        objs.append(obj)
        cmds.append([cc, *_flags(), *extra, "-c", os.path.join(CSRC, src), "-o", obj])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        for out in ex.map(run, cmds):
            if verbose and out.strip():
                print(out, file=sys.stderr)
    tmp = lib + f".{os.getpid()}.tmp"
    run([cc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
