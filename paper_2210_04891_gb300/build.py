"""Build libsie.so in-tree for sm_103a (nvcc + g++, no cmake).

Each translation unit is compiled in parallel; the library is linked beside
this file.  Host code is compiled without floating-point contraction so that
integer decisions taken from floating point (stencil nodes, near pairs) are
the same on x86-64 and aarch64 hosts.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsie.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU = ["sie_plan.cu", "sie_pfft.cu", "sie_near_mma.cu", "sie_solve.cu", "sie_noalloc.cu", "sie_plane.cu", "sie_batch.cu", "sie_tune.cu", "sie_learned.cu",
      "sie_lossy.cu", "sie_nd.cu", "sie_df.cu"]
CPP = ["sie_host.cpp"]


def nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsie")


def _sources():
    return [os.path.join(CSRC, f) for f in CU + CPP] + [
        os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))] + [
        os.path.join(INC, "sie.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force=False, verbose=False):
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    common = ["-O3", "-std=c++17", "-I", INC, "-Xcompiler", "-fPIC,-fopenmp,-ffp-contract=off"]
    jobs = []
    for f in CU:
        jobs.append([cc, *common, *ARCH, "-lineinfo", "-c", os.path.join(CSRC, f), "-o",
                     os.path.join(BUILD, f + ".o")])
    for f in CPP:
        jobs.append(["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-ffp-contract=off", "-I", INC, "-c",
                     os.path.join(CSRC, f), "-o", os.path.join(BUILD, f + ".o")])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(run, jobs))
    if verbose:
        print("".join(outs))
    objs = [os.path.join(BUILD, f + ".o") for f in CU + CPP]
    tmp = LIB + ".tmp"
    run([cc, "-shared", *ARCH, "-cudart", "shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
