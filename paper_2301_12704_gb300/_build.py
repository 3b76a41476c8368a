"""Build the in-tree CUDA library libaifmm.so for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked into a shared
library next to this file.  No PyTorch headers are involved: the library
exposes a plain C ABI (include/aifmm.h).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libaifmm.so")
SOURCES = ["api.cu", "tree.cu", "nnca.cu", "factor.cu", "solve.cu", "gmres.cu", "gemm.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _flags(debug: bool):
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"] + ARCH
    if os.environ.get("AIFMM_PTXAS_V"):
        f += ["-Xptxas", "-v"]
    return f


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every source that is newer than its object and link the .so."""
    os.makedirs(OUT, exist_ok=True)
    headers = [os.path.join(CSRC, x) for x in os.listdir(CSRC) if x.endswith((".h", ".cuh"))]
    headers.append(os.path.join(HERE, "..", "include", "aifmm.h"))
    headers.append(os.path.join(HERE, "..", "include", "aifmm_kernels.h"))
    hdr_time = max(os.path.getmtime(x) for x in headers)
    exe = nvcc()
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src.replace(".cu", ".o"))
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr_time):
            jobs.append([exe, "-c", s, "-o", o] + _flags(False))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for cmd, r in ex.map(run, jobs):
                if verbose or r.returncode:
                    sys.stderr.write(r.stdout + r.stderr)
                if r.returncode:
                    raise RuntimeError("nvcc failed: " + " ".join(cmd))
    if jobs or not os.path.exists(LIB):
        cmd = [exe, "-shared", "-o", LIB] + objs + ARCH + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
