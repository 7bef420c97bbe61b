"""Build the lbpf CUDA library (liblbpf.so) in-tree for sm_103a with nvcc.

One translation unit per lattice pair plus the host API and the
precision-generic kernels, compiled in parallel and linked into a shared
library beside this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build", platform.machine())  # objects of this host architecture only
LIB = os.path.join(HERE, "liblbpf.so")
SOURCES = ["lbpf_api.cu", "lbpf_fields.cu", "lbpf_d2q9.cu", "lbpf_d3q15.cu", "lbpf_d3q19.cu", "lbpf_d3q27.cu",
           "lbpf_static.cu", "lbpf_nn.cu", "lbpf_unet.cu"]
HEADERS = ["lbpf_internal.cuh", "step_kernel.cuh", "staged_kernel.cuh", "aux_kernels.cuh", "lbpf_nn.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"] + ARCH


def nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    include = os.path.join(os.path.dirname(HERE), "include")
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(include, "lbpf.h")]
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            jobs.append([nvcc()] + FLAGS + ["-I", include, "-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            res = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, res):
            if verbose or r.returncode:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    stamp = os.path.join(BUILD, "liblbpf.stamp")
    if force or jobs or _stale(LIB, objs) or _stale(stamp, [LIB]):
        tmp = LIB + f".tmp{os.getpid()}"
        r = subprocess.run([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"], capture_output=True, text=True)
        if r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, LIB)
        open(stamp, "w").write(platform.machine() + "\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
