"""Shared test helpers: build matching oracle and GPU runs of one workload.

Both sides receive the same seeded inputs (sizes, physical parameters,
seeds); each computes everything else itself.
"""
import numpy as np

ORC_LAT = {0: 0, 1: 1, 2: 2, 3: 3}


def oracle_run(O, lattice, shape, params, crystals, seeds=None, fields=None, grad=0, xi=1e-7, bc=0,
               adv=(0.0, 0.0, 0.0)):
    nz, ny, nx = shape
    prm = dict(params)
    lam = prm.pop("lam", None)
    p = O.make_params(ORC_LAT[lattice], nx, ny, nz, grad=grad, lam=lam, xi=xi,
                      crystals=[O.make_crystal(**c) for c in crystals], bc=bc, adv=adv, **prm)
    o = O.Oracle(p)
    if seeds is not None:
        o.seed([list(s) for s in seeds])
    else:
        o.set_fields(*fields)
    return o


def gpu_run(L, lattice, shape, params, crystals, seeds=None, fields=None, grad=0, precision=None, xi=1e-7,
            stream=None, bc=0, adv=(0.0, 0.0, 0.0)):
    nz, ny, nx = shape
    prm = dict(params)
    lam = prm.pop("lam", None)
    dom = L.make_domain(nx, ny, nz, lam=0.0 if lam is None else lam, xi=xi,
                        crystals=[L.make_crystal(**c) for c in crystals], bc=bc, adv=adv, **prm)
    s = L.Solver(dom, lattice, grad, L.LBPF_FP64 if precision is None else precision, stream=stream)
    if seeds is not None:
        s.seed(seeds)
    else:
        s.write_fields(*fields)
    return s


def maxabs(a, b):
    return float(np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)).max())
