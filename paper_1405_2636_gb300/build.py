"""Build ``libspx.so`` in-tree for sm_103a (nvcc + g++, no cmake).

Every translation unit is compiled in parallel into ``_build/`` next to this
file, then linked into ``libspx.so`` beside the package's Python files.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libspx.so")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", CSRC, "-I", INCLUDE]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-I", CSRC, "-I", INCLUDE]

CU_SOURCES = ["api.cu", "factor.cu", "solve.cu", "update_tc.cu", "batch_api.cu", "batch_lu.cu", "selinv.cu",
              "sweep.cu", "study.cu", "fqueue_f64.cu", "fqueue_tc.cu", "fqueue_ldlt.cu"]
CXX_SOURCES = ["analyze.cpp"]
HEADERS = ["kernels.cuh", "spx_plan.h", "batch_kernel.cuh", "operand.cuh", "blocks.cuh", "tc_common.cuh", "fqueue.cuh"]


def _sources():
    return [os.path.join(CSRC, f) for f in CU_SOURCES + CXX_SOURCES + HEADERS] + [
        os.path.join(INCLUDE, "spx.h"), os.path.abspath(__file__)]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    objs = []
    for f in CU_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        cmd = [NVCC] + NVCC_FLAGS + ["-c", os.path.join(CSRC, f), "-o", obj]
        jobs.append((cmd, f))
        objs.append(obj)
    for f in CXX_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        cmd = ["g++"] + CXX_FLAGS + ["-c", os.path.join(CSRC, f), "-o", obj]
        jobs.append((cmd, f))
        objs.append(obj)
    procs = []
    for cmd, name in jobs:
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), name))
    failed = []
    for p, name in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append(f"--- {name} ---\n{out.decode(errors='replace')}")
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        raise RuntimeError("libspx build failed:\n" + "\n".join(failed))
    tmp = LIB + f".tmp{os.getpid()}"
    link = [NVCC] + ARCH + ["-shared", "-Xlinker", "--no-undefined", "-o", tmp] + objs
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("libspx link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
