"""Build step of libprism_proj: nvcc for sm_103a, in-tree output.

``python -m paper_2608_25666_b300.build`` (or ``build()``) compiles
``csrc/*.cu``, ``csrc/prism_server.cpp`` into ``_build/libprism_proj.so``.  nvcc cross-compiles
without a GPU, so this runs on any machine with the CUDA toolkit.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

_HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(_HERE)
SRC = os.path.join(_HERE, "csrc", "prism_proj.cu")
SRC_SERVER = os.path.join(_HERE, "csrc", "prism_server.cpp")
SRC_MPPI = os.path.join(_HERE, "csrc", "prism_mppi.cu")
SRC_WS = os.path.join(_HERE, "csrc", "prism_ws.cu")
SOURCES = [SRC, SRC_MPPI, SRC_SERVER, SRC_WS]
HEADERS = [os.path.join(_HERE, "csrc", "tcgen05_common.cuh")]
HDR = os.path.join(ROOT, "include", "prism_proj.h")
OUT = os.path.join(_HERE, "_build", "libprism_proj.so")

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    newest = max([os.path.getmtime(f) for f in SOURCES + HEADERS] + [os.path.getmtime(HDR)])
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= newest:
        return OUT
    tmp = OUT + f".tmp{os.getpid()}"
    cmd = [nvcc(), *NVCC_FLAGS, "-I", os.path.join(ROOT, "include"), "-o", tmp, *SOURCES, "-lpthread"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
