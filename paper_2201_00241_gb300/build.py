"""Build librh.so (CUDA for sm_103a + host C++) in-tree under _build/.

nvcc compiles the .cu translation units with ``-gencode arch=compute_103a,code=sm_103a``;
g++ compiles the host symbolic phase; the pieces compile in parallel and are
linked with nvcc into a shared library loaded by ``paper_2201_00241_gb300.rh``.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "librh.so")
# the same sources with every device index check on (-DRH_BOUNDS): a failed check sets an
# error word that rh_bounds_check reads, and the access is skipped
LIB_BOUNDS = os.path.join(OUT, "librh_bounds.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

CU = ["kernels.cu", "dense.cu", "api.cu", "peak.cu"]
CPP = ["symbolic.cpp"]
HEADERS = ["rh_internal.h", "rh_kernels.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _sources():
    return [os.path.join(CSRC, f) for f in CU + CPP + HEADERS] + [os.path.join(INCLUDE, "rh.h")]


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    lib = LIB_BOUNDS if bounds else LIB
    tag = ".bounds" if bounds else ""
    if not force and os.path.exists(lib):
        t = os.path.getmtime(lib)
        if all(os.path.getmtime(s) <= t for s in _sources()):
            return lib
    nvcc = _nvcc()
    procs = []
    objs = []
    for f in CU:
        o = os.path.join(OUT, f + tag + ".o")
        objs.append(o)
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
               *(["-DRH_BOUNDS"] if bounds else []), "-c", os.path.join(CSRC, f), "-o", o]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for f in CPP:
        o = os.path.join(OUT, f + tag + ".o")
        objs.append(o)
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-I", INCLUDE, "-c", os.path.join(CSRC, f), "-o", o]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            print(" ".join(cmd))
            print(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(cmd[-3])
    if failed:
        raise RuntimeError(f"compilation failed: {failed}")
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
    print(build(force=True, verbose=True, bounds=True))
