"""Build the GP-MOOD CUDA library (libgpmood.so) for sm_103a, in-tree.

Translation units are compiled in parallel: the host driver with the
precision-independent kernels, one file per precision for the stage kernels,
and the binary128 weight solver (plain C, gcc).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libgpmood.so")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-prec-div=true", "-prec-sqrt=true", "-ftz=false"]
CUDA_SOURCES = ["gpmood_api.cu", "gpmood_batch.cu", "kernels_f64.cu", "kernels_f32.cu"]
C_SOURCES = ["gp_weights.c"]


def nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgpmood")
    return cand


def _sources():
    return [os.path.join(CSRC, f) for f in CUDA_SOURCES + C_SOURCES] + [
        os.path.join(CSRC, f)
        for f in os.listdir(CSRC)
        if f.endswith((".cuh", ".h"))
    ] + [os.path.join(INCLUDE, "gpmood.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def _compile(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stderr


def build(force=False, verbose=False, ptxas_info=False):
    """Compile and link libgpmood.so; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nv = nvcc()
    jobs = []
    objs = []
    for f in CUDA_SOURCES:
        o = os.path.join(OUT, f + ".o")
        cmd = [nv, *ARCH, *NVCC_FLAGS, "-I", INCLUDE, "-c", os.path.join(CSRC, f), "-o", o]
        if ptxas_info:
            cmd += ["-Xptxas", "-v"]
        jobs.append(cmd)
        objs.append(o)
    for f in C_SOURCES:
        o = os.path.join(OUT, f + ".o")
        jobs.append(["gcc", "-O2", "-std=c11", "-fPIC", "-c", os.path.join(CSRC, f), "-o", o])
        objs.append(o)
    logs = []
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        for log in ex.map(_compile, jobs):
            logs.append(log)
    tmp = LIB + f".tmp{os.getpid()}"
    _compile([nv, *ARCH, "-shared", "-o", tmp, *objs, "-lm"])
    os.replace(tmp, LIB)
    if verbose or ptxas_info:
        print("\n".join(l for l in logs if l))
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force=True, ptxas_info="-v" in sys.argv))
