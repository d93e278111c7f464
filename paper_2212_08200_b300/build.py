"""Builds libgg.so (the CUDA library behind include/gg.h) in-tree with nvcc
for sm_103a.  Run `python -m paper_2212_08200_b300.build` or call build()."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libgg.so")
OBJDIR = os.path.join(ROOT, "_build", "gg")

SOURCES = ["gg_api.cu", "gg_graph.cu", "gg_bsp.cu", "gg_async.cu", "gg_noalloc.cu", "gg_batch.cu", "gg_multi.cu", "gg_server.cu", "gg_tune.cu", "gg_edge.cu", "gg_part.cu"]
HEADERS = ["gg_common.cuh", "gg_host.h", "gg_multi.h"]

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O3", "-I" + INCLUDE, "-I" + CSRC,
         "--expt-relaxed-constexpr"] + os.environ.get("GG_NVCC_EXTRA", "").split()


def _newest_dep() -> float:
    paths = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "gg.h"), __file__]
    return max(os.path.getmtime(p) for p in paths if os.path.exists(p))


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(OBJDIR, exist_ok=True)
    dep = _newest_dep()
    objs = []
    changed = force or not os.path.exists(LIB)
    for src in SOURCES:
        sp = os.path.join(CSRC, src)
        op = os.path.join(OBJDIR, src.replace(".cu", ".o"))
        objs.append(op)
        if force or not os.path.exists(op) or os.path.getmtime(op) < max(os.path.getmtime(sp), dep):
            cmd = [NVCC, *ARCH, *FLAGS, "-c", sp, "-o", op]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            subprocess.check_call(cmd)
            changed = True
    if changed:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas-info" in sys.argv)
    print(LIB)
