"""Build the native library libstc.so in-tree (nvcc for sm_103a + g++ for the host analysis).

    python -m paper_2609_29765_gb300.build

The shared library exports the C ABI declared in include/stc.h.  No PyTorch headers are
involved: the Python side talks to it through ctypes.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INC = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libstc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

SOURCES_CU = ["replay.cu", "compose.cu"]
SOURCES_CPP = ["analyze.cpp", "supernodal.cpp", "plan_io.cpp"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _sources():
    return [os.path.join(CSRC, s) for s in SOURCES_CU + SOURCES_CPP] + \
        [os.path.join(CSRC, "plan.hpp"), os.path.join(INC, "stc.h")]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(verbose: bool = False) -> str:
    """Compile every translation unit (in parallel) and link libstc.so."""
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    cmds = []
    objs = []
    for s in SOURCES_CU:
        o = os.path.join(OUT, s + ".o")
        objs.append(o)
        cmds.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", INC, "-c", os.path.join(CSRC, s), "-o", o])
    for s in SOURCES_CPP:
        o = os.path.join(OUT, s + ".o")
        objs.append(o)
        cmds.append(["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-I", INC, "-c",
                     os.path.join(CSRC, s), "-o", o])

    def run(c):
        if verbose:
            print(" ".join(c), flush=True)
        r = subprocess.run(c, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(c), r.stdout, r.stderr))
        return r

    with ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        list(ex.map(run, cmds))
    tmp = LIB + ".tmp%d" % os.getpid()
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
