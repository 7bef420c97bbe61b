"""The staged step kernel (rows brought to shared memory by bulk asynchronous
copies) against the generic kernel and the FP64 oracle.

The staged kernel runs the same arithmetic as the generic one; only its data
movement differs.  It is chosen by the environment variable
LBPF_KERNEL=staged at context creation, for 3D D3Q15/D3Q19 domains with
16-bit deviation storage whose nx is a multiple of 8 and at least 64.  Two
independent data paths that agree bit for bit also cross-check each other.
"""
import os

import numpy as np
import pytest

from helpers import gpu_run, maxabs, oracle_run
from paper_1606_09432_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1606_09432_gb300 import build as B
    from paper_1606_09432_gb300 import lbpf
    B.build()
    lbpf.load()
    return lbpf


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


def run_kernel(L, kernel, lattice, shape, params, crystals, seeds=None, fields=None, precision=2, steps=0,
               schedule=None):
    old = os.environ.get("LBPF_KERNEL")
    os.environ["LBPF_KERNEL"] = kernel
    try:
        s = gpu_run(L, lattice, shape, params, crystals, seeds=seeds, fields=fields, precision=precision)
    finally:
        if old is None:
            del os.environ["LBPF_KERNEL"]
        else:
            os.environ["LBPF_KERNEL"] = old
    if schedule:
        L.lbpf_set_schedule(s.ctx, *schedule)
    s.step(steps)
    return s


C3P = dict(W.C3D_PARAMS, delta=0.4)


@pytest.mark.parametrize("precision", [2, 3, 4])
@pytest.mark.parametrize("lattice,shape", [(1, (30, 40, 72)), (2, (17, 24, 96)), (1, (5, 9, 64))])
def test_staged_matches_generic(L, lattice, shape, precision):
    """Ragged tiles in x and y, a row crossing the periodic x edge in every
    tile row, segments of one plane: the two kernels agree."""
    nz, ny, nx = shape
    seeds = [(nx * 0.43, ny * 0.55, nz * 0.5, 6.0, 0)]
    cr = [dict(kind=3, eps=0.02, gamma=-0.02)]
    a = run_kernel(L, "staged", lattice, shape, C3P, cr, seeds=seeds, precision=precision, steps=60)
    b = run_kernel(L, "generic", lattice, shape, C3P, cr, seeds=seeds, precision=precision, steps=60)
    assert a.query(L.LBPF_Q_KERNEL) == 1 and b.query(L.LBPF_Q_KERNEL) == 0
    pa, ua = a.fields()
    pb, ub = b.fields()
    print(f"staged vs generic {shape} lattice {lattice} precision {precision}: phi {maxabs(pa, pb):.2e}, "
          f"u {maxabs(ua, ub):.2e}, identical {np.array_equal(pa, pb) and np.array_equal(ua, ub)}")
    assert maxabs(pa, pb) <= 1e-5 and maxabs(ua, ub) <= 1e-5
    ga, gb = a.populations(0), b.populations(0)
    assert maxabs(ga, gb) <= 1e-5
    # one-plane segments and the other segment lengths give the same result
    c = run_kernel(L, "staged", lattice, shape, C3P, cr, seeds=seeds, precision=precision, steps=60,
                   schedule=(8, 1))
    assert np.array_equal(c.fields()[0], pa) and np.array_equal(c.fields()[1], ua)


def test_staged_vs_oracle_c3_crop(L, O):
    """64^3 <110> crop of the 512^3 configuration, FP16 deviations through the
    staged kernel, against the FP64 oracle after 500 steps (the 16-bit error
    is stated, with the sanity bounds of the generic kernel's test)."""
    w = W.c3(64, eps=0.0, gamma=-0.02)
    cr = [w["aniso"]]
    o = oracle_run(O, 1, w["shape"], w["params"], cr, seeds=w["seeds"])
    s = run_kernel(L, "staged", 1, w["shape"], w["params"], cr, seeds=w["seeds"], precision=2)
    assert s.query(L.LBPF_Q_KERNEL) == 1
    _, _, c0 = s.measure(*w["centre"])
    o.step(500)
    s.step(500)
    phi, u = s.fields()
    ophi, ou, _ = o.fields()
    tip, _, c1 = s.measure(*w["centre"])
    otip = o.measure(*w["centre"])[0]
    e = (maxabs(phi, ophi), maxabs(u, ou), float(np.abs(tip - otip).max()))
    print(f"staged FP16 deviations vs FP64 oracle, 64^3, 500 steps: phi {e[0]:.2e}, u {e[1]:.2e}, tips {e[2]:.2e}, "
          f"drift {abs(c1 - c0) / abs(c0):.2e}")
    assert e[0] < 1.0 and e[1] < 0.5 and e[2] < 1.0
    assert abs(c1 - c0) <= 1e-5 * abs(c0)


def test_staged_full_size_sampled(L, O):
    """512^3 D3Q15 FP16 deviations, the benchmark's configuration and launch
    (staged kernel, autotuned schedule), two steps, against the FP64 oracle
    on sampled sites: after k steps a site depends only on the initial state
    within 2k + 2 sites, so a 32^3 periodic crop centred on the sample, seeded
    alike, gives the exact values in its central 16^3."""
    n, k, m = 512, 2, 32
    w = W.c3(n, eps=0.0, gamma=-0.02)
    cr = [w["aniso"]]
    s = run_kernel(L, "staged", 1, w["shape"], w["params"], cr, seeds=w["seeds"], precision=2)
    assert s.query(L.LBPF_Q_KERNEL) == 1
    s.step(k)
    phi, u = s.fields()
    c = n // 2
    for centre in [(c + 8, c, c), (c + 3, c + 5, c - 6), (c, c, c), (40, 300, 500)]:
        sx, sy, sz = centre
        dx_, dy_, dz_ = (w["seeds"][0][0] - sx, w["seeds"][0][1] - sy, w["seeds"][0][2] - sz)
        if max(abs(dx_), abs(dy_), abs(dz_)) <= m // 2 - 4:
            seeds = [(dx_ + m // 2, dy_ + m // 2, dz_ + m // 2, w["seeds"][0][3], 0)]
        else:  # far from the nucleus: phi = -1 on the whole crop (a seed of negative radius)
            seeds = [(m // 2, m // 2, m // 2, -100.0, 0)]
        o = oracle_run(O, 1, (m, m, m), w["params"], cr, seeds=seeds)
        o.step(k)
        ophi, ou, _ = o.fields()
        lo, hi = m // 2 - 8, m // 2 + 8
        sl = (slice(sz - 8, sz + 8), slice(sy - 8, sy + 8), slice(sx - 8, sx + 8))
        ep, eu = maxabs(phi[sl], ophi[lo:hi, lo:hi, lo:hi]), maxabs(u[sl], ou[lo:hi, lo:hi, lo:hi])
        print(f"512^3 after {k} steps, 16^3 sample at {centre}: phi {ep:.2e}, u {eu:.2e}")
        assert ep <= 1e-3 and eu <= 1e-3
