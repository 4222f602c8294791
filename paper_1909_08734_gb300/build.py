"""Build the in-tree shared library libcpm_gb300.so for sm_103a (GB300).

Host set-up code is compiled with g++ (-ffp-contract=off keeps every set-membership
decision reproducible); device code with nvcc for sm_103a only.  Objects go to
``_build/``; the library lands next to this file.  No CMake, no torch extension
machinery: the result is a plain C-ABI shared object.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcpm_gb300.so")
INCLUDE = os.path.join(ROOT, "include")

HOST_SRC = ["host/band.cpp", "host/partition.cpp", "host/local_coo.cpp", "host/ordering.cpp", "capi_host.cpp"]
CUDA_SRC = ["cuda/apply.cu", "cuda/factor.cu", "cuda/lu_tc.cu", "cuda/trsv.cu", "cuda/krylov.cu",
            "cuda/stationary.cu", "cuda/selftest.cu", "cuda/probe.cu", "cuda/band_dev.cu", "capi_device.cu",
            "noalloc.cu"]
# set decisions (closest points, tube test, weights) computed on the device must match the host
# code bit for bit: no floating-point contraction there
NO_FMAD = {"cuda/band_dev.cu"}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def _obj(src: str) -> str:
    return os.path.join(BUILD, src.replace("/", "_") + ".o")


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    headers = [os.path.join(INCLUDE, "cpm.h")]
    for d, _, fs in os.walk(CSRC):
        headers += [os.path.join(d, f) for f in fs if f.endswith((".h", ".cuh"))]
    jobs = []
    for src in HOST_SRC:
        s = os.path.join(CSRC, src)
        o = _obj(src)
        if _stale(o, [s] + headers):
            jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-fopenmp", "-ffp-contract=off",
                         "-Wall", "-Wno-unknown-pragmas", "-I", INCLUDE, "-c", s, "-o", o])
    for src in CUDA_SRC:
        s = os.path.join(CSRC, src)
        o = _obj(src)
        if _stale(o, [s] + headers):
            cmd = [nvcc, "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler",
                   "-fPIC,-fopenmp,-ffp-contract=off", "-I", INCLUDE, "-c", s, "-o", o]
            if src in NO_FMAD:
                cmd.insert(1, "-fmad=false")
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    logs = []
    with cf.ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        for out in ex.map(_run, jobs):
            logs.append(out)
    objs = [_obj(s) for s in HOST_SRC + CUDA_SRC]
    if jobs or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        _run([nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp",
              "-cudart", "shared", "-L", os.path.join(cuda, "lib64"),
              "-Xlinker", "-rpath," + os.path.join(cuda, "lib64")])
        os.replace(tmp, LIB)
    if verbose:
        for line in logs:
            if line.strip():
                print(line)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="--ptxas" in sys.argv))
