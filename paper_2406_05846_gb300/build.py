"""Build libstrom.so in-tree for sm_103a (nvcc for CUDA sources, g++ for host C++)."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libstrom.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU = ["psd.cu", "factor.cu", "admm.cu", "solver.cu", "serve.cu", "noalloc.cu", "warm.cu", "sparse.cu",
      "sparse_solver.cu", "server.cu"]
CPP = ["relax.cpp", "capi.cpp", "certify.cpp", "warm_select.cpp", "sdp_import.cpp", "rank_test.cpp", "sparse_sym.cpp"]


def _nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libstrom")
    return p


def _sources_mtime():
    t = 0.0
    for f in os.listdir(CSRC):
        t = max(t, os.path.getmtime(os.path.join(CSRC, f)))
    t = max(t, os.path.getmtime(os.path.join(HERE, "..", "include", "strom.h")))
    t = max(t, os.path.getmtime(__file__))
    return t


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources_mtime():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    # host code is compiled without FMA contraction so that x86 and Arm
    # builds give bit-identical host results
    for f in CU:
        o = os.path.join(BUILD, f + ".o")
        jobs.append([nvcc, *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "-c", os.path.join(CSRC, f), "-o", o])
    for f in CPP:
        o = os.path.join(BUILD, f + ".o")
        jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-Wall", "-ffp-contract=off", "-I/usr/local/cuda/include",
                     "-c", os.path.join(CSRC, f), "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(BUILD, f + ".o") for f in CU + CPP]
    tmp = LIB + ".tmp"
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
