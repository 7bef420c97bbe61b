"""CPU checks of the C ABI: the library loads, exports every function that
include/lbpf.h declares, and rejects invalid arguments before touching the
GPU.  No compute call is made."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lbpf_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    from paper_1606_09432_gb300 import build as B
    from paper_1606_09432_gb300 import lbpf
    B.build()
    return lbpf


def test_exports_every_declared_symbol(L):
    lib = L.load()
    decl = declared_functions()
    assert len(decl) >= 10
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(L.EXPORTED) == decl


def test_invalid_arguments_rejected_before_gpu(L):
    d = L.make_domain(1, 8, 1, dx=1, dt=0.1, W0=1, tau0=1, kappa=1)
    for args in [(d, 0, 0, 0), (L.make_domain(8, 8, 1, dx=1, dt=0.1, W0=1, tau0=1, kappa=1), 7, 0, 0),
                 (L.make_domain(8, 8, 1, dx=1, dt=0.1, W0=1, tau0=1, kappa=1), 0, 0, 9),
                 (L.make_domain(8, 8, 1, dx=1, dt=-0.1, W0=1, tau0=1, kappa=1), 0, 0, 0),
                 (L.make_domain(8, 8, 4, dx=1, dt=0.1, W0=1, tau0=1, kappa=1), 0, 0, 0)]:
        with pytest.raises(L.LbpfError) as e:
            L.lbpf_create([args[0]], args[1], args[2], args[3])
        assert e.value.code == L.LBPF_EINVAL
        assert L.lbpf_last_error(None)


def test_invalid_velocity_rejected_before_gpu(L):
    """The advective heat equilibrium: no z component on a 2D lattice,
    tangential to walls, finite."""
    def dom(nz=1, bc=0, adv=(0.1, 0.0, 0.0)):
        return L.make_domain(8, 8, nz, dx=1, dt=0.1, W0=1, tau0=1, kappa=1, bc=bc, adv=adv)
    cases = [(dom(adv=(0, 0, 0.1)), L.LBPF_D2Q9_D2Q5, L.LBPF_FP32_FP16DEV),
             (dom(adv=(0, 0, 0.1)), L.LBPF_D2Q9_D2Q5, L.LBPF_FP64),
             (dom(bc=L.LBPF_BC_WALL_X), L.LBPF_D2Q9_D2Q5, L.LBPF_FP64),
             (dom(nz=8, bc=L.LBPF_BC_WALL_Z, adv=(0.1, 0.0, 0.2)), L.LBPF_D3Q15_D3Q7, L.LBPF_FP32),
             (dom(adv=(float("nan"), 0, 0)), L.LBPF_D2Q9_D2Q5, L.LBPF_FP64)]
    for d, lat, prec in cases:
        with pytest.raises(L.LbpfError) as e:
            L.lbpf_create([d], lat, L.LBPF_GRAD_DD, prec)
        assert e.value.code == L.LBPF_EINVAL


def test_null_context_is_safe(L):
    lib = L.load()
    assert lib.lbpf_destroy(None) == 0
    assert lib.lbpf_step(None, 1) == L.LBPF_EINVAL
