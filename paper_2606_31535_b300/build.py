"""Builds libpeers.so (the C-ABI library: host analysis + CUDA kernels for sm_103a) in-tree,
and its bounds-checked variant libpeers_bounds.so (compiled with PEERS_BOUNDS=1: every
kernel access to a panel, front, carry, relative map or result is checked against the extent
the analysis computed, and a violation sets the call's error flag and skips the access).

    python -m paper_2606_31535_b300.build [--force] [--bounds]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpeers.so")
BUILD_BOUNDS = os.path.join(HERE, "_build_bounds")
LIB_BOUNDS = os.path.join(HERE, "libpeers_bounds.so")
SOURCES = ["analyze.cpp", "factor.cu", "sweep.cu", "peaks.cu", "sweep_static.cu", "batch.cu", "serve.cu", "autotune.cu", "blockinv.cu", "sparsify.cu", "capi.cu"]
HEADERS = ["internal.h", "device.cuh", "handles.h"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O3,-Wall",
         "-I", CSRC, "-I", os.path.join(ROOT, "include")]


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    """Compiles the changed sources and links the library; returns its path.  bounds=True
    builds the bounds-checked variant into its own directory and file."""
    build_dir, lib = (BUILD_BOUNDS, LIB_BOUNDS) if bounds else (BUILD, LIB)
    flags = FLAGS + (["-DPEERS_BOUNDS=1"] if bounds else [])
    os.makedirs(build_dir, exist_ok=True)
    hdr = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "peers.h"),
                                                     os.path.abspath(__file__)]
    hdr_time = _newest(hdr)
    jobs = []
    objs = []
    for src in SOURCES:
        sp = os.path.join(CSRC, src)
        obj = os.path.join(build_dir, src + ".o")
        objs.append(obj)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(hdr_time, os.path.getmtime(sp)):
            cmd = [NVCC] + ARCH + flags + ["-c", sp, "-o", obj]
            if src.endswith(".cpp"):
                cmd = [NVCC] + flags + ["-x", "c++", "-c", sp, "-o", obj]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or r.returncode != 0:
                sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {cmd[-3]}")
    if force or jobs or not os.path.exists(lib) or os.path.getmtime(lib) < _newest(objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                bounds="--bounds" in sys.argv))
