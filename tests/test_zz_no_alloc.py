"""lbpf_field_sums_static: the measurement sums without any device allocation.

Some callers cannot let a library allocate device memory when they call it
(their own pool allocator owns the device memory, or cudaMalloc's implicit
synchronisation is not acceptable in their loop).  They call this entry point
with their own phi, u and output buffers; its scratch is a fixed device array
inside the library.  This test checks it, through the C ABI, against the sums
that lbpf_measure (which uses scratch allocated by its context) reports, on
two consecutive calls, in FP64 and FP32.  The file is named so that pytest
collects it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_static_sums_match_measure(precision):
    import torch

    from paper_1606_09432_gb300 import build as B
    from paper_1606_09432_gb300 import lbpf as L
    from paper_1606_09432_gb300 import workloads as W

    B.build()
    w = W.c2(40)
    prm = dict(w["params"])
    lam = prm.pop("lam")
    dom = L.make_domain(40, 40, 40, lam=lam, crystals=[L.make_crystal(**w["aniso"])], **prm)
    s = L.Solver(dom, L.LBPF_D3Q15_D3Q7, L.LBPF_GRAD_DD, precision)
    s.seed(w["seeds"])
    n = 40 ** 3
    tdt = torch.float64 if precision == L.LBPF_FP64 else torch.float32
    for call in range(2):
        s.step(30)
        _, sf, cs = s.measure(*w["centre"])
        phi = torch.empty((40, 40, 40), dtype=tdt, device="cuda")
        u = torch.empty((40, 40, 40), dtype=tdt, device="cuda")
        L.lbpf_read_field(s.ctx, 0, L.LBPF_FIELD_PHI, phi)
        L.lbpf_read_field(s.ctx, 0, L.LBPF_FIELD_U, u)
        out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        L.lbpf_field_sums_static(phi, u, precision, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert abs(o[0] / n - sf) <= 1e-12 * abs(sf), (call, o[0] / n, sf)
        assert abs(o[1] - cs) <= 1e-12 * abs(cs), (call, o[1], cs)
        assert o[2] == 0.0
    s.close()


def test_static_sums_reject_oversize():
    import ctypes as C

    from paper_1606_09432_gb300 import lbpf as L

    lib = L.load()
    one = C.c_double(0.0)
    p = C.cast(C.pointer(one), C.c_void_p)
    # sizes are checked before any device work
    assert lib.lbpf_field_sums_static(p, p, 268435456 + 1, 0, p, None) == L.LBPF_ERANGE
    assert lib.lbpf_field_sums_static(p, p, 0, 0, p, None) == L.LBPF_ERANGE
    assert lib.lbpf_field_sums_static(None, p, 10, 0, p, None) == L.LBPF_EINVAL
