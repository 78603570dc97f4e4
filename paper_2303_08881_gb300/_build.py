"""Build libilu2l.so in-tree: every CUDA translation unit compiled for sm_103a with
nvcc (in parallel), the host setup with g++ (no floating-point contraction), linked
into ``paper_2303_08881_gb300/libilu2l.so``. Objects go to ``_build/`` at the repo root."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INC = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "libilu2l.so")
BUILD = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU = ["capi.cu", "kernels_apply.cu", "kernels_ilu.cu", "kernels_krylov.cu", "kernels_stream.cu", "noalloc.cu",
      "probes.cu", "kernels_ilut.cu"]
CPP = ["setup_host.cpp"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libilu2l.so")
    return cand


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INC, "ilu2l.h")]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= _deps():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ["-std=c++17", "-O3", "-I", INC, "-I", CSRC]
    jobs = []
    for f in CU:
        obj = os.path.join(BUILD, f + ".o")
        jobs.append([nvcc, *ARCH, "-lineinfo", *common, "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "-c", os.path.join(CSRC, f), "-o", obj])
    for f in CPP:
        obj = os.path.join(BUILD, f + ".o")
        jobs.append(["g++", *common, "-fPIC", "-ffp-contract=off", "-pthread",
                     "-I", os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include"),
                     "-c", os.path.join(CSRC, f), "-o", obj])

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + p.stdout + p.stderr)
        if verbose and (p.stdout or p.stderr):
            print(p.stdout + p.stderr, file=sys.stderr)
        return cmd[-1]

    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(run, jobs))
    tmp = OUT + f".{os.getpid()}.tmp"
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-pthread"])
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
