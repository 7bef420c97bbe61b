"""lbpf_field_sums_static: the measurement sums without any device allocation.

Some callers cannot let a library allocate device memory when they call it
(their own pool allocator owns the device memory, or cudaMalloc's implicit
synchronisation is not acceptable in their loop).  They call this entry point
with their own phi, u and output buffers; its scratch is a fixed device array
inside the library, shared by every call.

The checks go through the C ABI and compare with FP64 sums computed on the
host, by NumPy, from the same phi and u copied back: on a field spanning
several of the kernel's 65,536-site chunks with a partial last chunk, then on
a smaller prefix of it (slots left over from the larger call must not leak
into the result), then again on the whole field after more steps, for every
precision.  The sums of lbpf_measure (scratch owned by its context) must agree
too.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N_SIDE = 96                    # 884,736 sites: 13 full chunks and a partial one
PREFIX = 65537                 # two chunks, the second holding one site


def host_sums(phi, u):
    p = np.asarray(phi, dtype=np.float64).ravel()
    v = np.asarray(u, dtype=np.float64).ravel()
    terms_sf = 0.5 * (1.0 + p)
    terms_cs = v - 0.5 * p
    return terms_sf.sum(), terms_cs.sum(), np.abs(terms_sf).sum(), np.abs(terms_cs).sum()


@pytest.mark.parametrize("precision", [0, 1, 2, 3, 4])
def test_static_sums_match_host_fp64(precision):
    import torch

    from paper_1606_09432_gb300 import build as B
    from paper_1606_09432_gb300 import lbpf as L
    from paper_1606_09432_gb300 import workloads as W

    B.build()
    n = N_SIDE
    w = W.c2(n)
    prm = dict(w["params"])
    lam = prm.pop("lam")
    dom = L.make_domain(n, n, n, lam=lam, crystals=[L.make_crystal(**w["aniso"])], **prm)
    s = L.Solver(dom, L.LBPF_D3Q15_D3Q7, L.LBPF_GRAD_DD, precision)
    s.seed(w["seeds"])
    tdt = torch.float64 if precision == L.LBPF_FP64 else torch.float32
    phi = torch.empty((n, n, n), dtype=tdt, device="cuda")
    u = torch.empty((n, n, n), dtype=tdt, device="cuda")
    out = torch.empty((3,), dtype=torch.float64, device="cuda")

    def call(count):
        out.fill_(float("nan"))
        L.lbpf_field_sums_static(phi.view(-1)[:count], u.view(-1)[:count], precision, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    for k, count in enumerate([n ** 3, PREFIX, n ** 3]):
        if k != 1:
            s.step(30)
            L.lbpf_read_field(s.ctx, 0, L.LBPF_FIELD_PHI, phi)
            L.lbpf_read_field(s.ctx, 0, L.LBPF_FIELD_U, u)
        o = call(count)
        sf, cs, asf, acs = host_sums(phi.view(-1)[:count].cpu().numpy(), u.view(-1)[:count].cpu().numpy())
        assert abs(o[0] - sf) <= 1e-12 * asf, (k, count, o[0], sf)
        assert abs(o[1] - cs) <= 1e-12 * acs, (k, count, o[1], cs)
        assert o[2] == 0.0
        if count == n ** 3:
            _, msf, mcs = s.measure(*w["centre"])
            assert abs(o[0] / count - msf) <= 1e-12 and abs(o[1] - mcs) <= 1e-12 * acs

    # a non-finite value is counted and left out of both sums
    phi.view(-1)[12345] = float("nan")
    o = call(PREFIX)
    ph = phi.view(-1)[:PREFIX].cpu().numpy().astype(np.float64)
    uu = u.view(-1)[:PREFIX].cpu().numpy().astype(np.float64)
    ok = np.isfinite(ph)
    sf, cs, asf, acs = host_sums(ph[ok], uu[ok])
    assert o[2] == 1.0 and abs(o[0] - sf) <= 1e-12 * asf and abs(o[1] - cs) <= 1e-12 * acs
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
    assert lib.lbpf_field_sums_static(p, p, 10, 9, p, None) == L.LBPF_EINVAL
