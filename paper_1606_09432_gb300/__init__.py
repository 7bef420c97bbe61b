"""lbpf: lattice Boltzmann phase-field crystal growth on one NVIDIA GB300.

The solver is the CUDA library liblbpf.so behind the C ABI of include/lbpf.h;
this package holds its sources (csrc/), the in-tree build (build.py), the
ctypes binding (lbpf.py) and seeded synthetic workloads (workloads.py).
"""
from . import lbpf  # noqa: F401
from .lbpf import Solver  # noqa: F401
