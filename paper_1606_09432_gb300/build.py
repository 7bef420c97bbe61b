"""Build the lbpf CUDA library (liblbpf.so) in-tree for sm_103a with nvcc.

The step and per-lattice kernels come from csrc/lbpf_lattice.cu compiled once
per lattice pair and storage precision (-DLBPF_LAT, -DLBPF_PREC); with the
host API, the dispatch table and the precision-generic kernels these objects
are compiled in parallel and linked into a shared library beside this file.
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
SOURCES = ["lbpf_api.cu", "lbpf_fields.cu", "lbpf_launchers.cu", "lbpf_static.cu", "lbpf_nn.cu", "lbpf_unet.cu"]
# (object name, source, extra flags): one lattice object per pair and precision
LATTICE_OBJECTS = [(f"lbpf_lattice_l{lat}_p{prec}", "lbpf_lattice.cu", [f"-DLBPF_LAT={lat}", f"-DLBPF_PREC={prec}"])
                   for lat in range(4) for prec in range(5)]
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
    units = [(src.replace(".cu", ""), src, []) for src in SOURCES] + LATTICE_OBJECTS
    for name, src, extra in units:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, name + ".o")
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            jobs.append([nvcc()] + FLAGS + extra + ["-I", include, "-c", s, "-o", o])
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
