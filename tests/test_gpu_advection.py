"""The advection-diffusion form of the heat scheme (Sec. 3.1) on the GPU
against the FP64 oracle: a uniform velocity v turns the heat equilibrium into
f_i^(0) = w_i u (1 + e_i . v dt / (e^2 dx)) (include/lbpf.h, lbpf_domain.adv).

The oracle's form is pinned on the CPU (its moments, the exact Fourier
propagator, the continuum phase speed and decay).  Here the CUDA path must
match it element by element, with the fields read between chunks of steps,
so that the lagged heat update (heat_sync), the load launch that follows it
and the replayed 16-step graphs all carry the advective term: FP64 within
1e-10 on phi and u, FP32 within 1e-4, the 16-bit deviation forms within
1e-4 (FP16) and 1e-3 (BF16, stochastic rounding).
"""
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


P3 = dict(W.C3D_PARAMS, delta=0.25)
P2 = dict(W.C4_PARAMS, delta=0.35)
# v dt / dx = (0.06, -0.0375, 0.0225) with the 3D parameters, (0.06, -0.04) in 2D
V3 = (40.0, -25.0, 15.0)
V2 = (60.0, -40.0, 0.0)


def compare_chunks(o, s, chunks, bar):
    for n in chunks:
        o.step(n)
        s.step(n)
        ophi, ou, _ = o.fields()
        phi, u = s.fields()
        e = (maxabs(phi, ophi), maxabs(u, ou))
        assert e[0] <= bar and e[1] <= bar, (n, e)
    return e


@pytest.mark.parametrize("lattice", [1, 2, 3])
def test_fp64_3d_advective_growth(L, O, lattice):
    """A <110> crystal grown in a uniform flow on a ragged periodic box; the
    heat populations too (D3Q15)."""
    shape = (19, 22, 37)
    cr = [dict(kind=3, eps=0.0, gamma=-0.02)]
    seeds = [(18.0, 11.0, 9.0, 6.0, 0)]
    o = oracle_run(O, lattice, shape, P3, cr, seeds=seeds, adv=V3)
    s = gpu_run(L, lattice, shape, P3, cr, seeds=seeds, adv=V3)
    compare_chunks(o, s, (7, 40, 33), 1e-10)
    if lattice == 1:
        og, of = o.populations()
        assert maxabs(s.populations(0), og) <= 1e-12 and maxabs(s.populations(1), of) <= 1e-12


@pytest.mark.parametrize("grad", [0, 1])
def test_fp64_2d_advective_growth(L, O, grad):
    """A fourfold 2D crystal in a flow, ragged strip tiles, both gradient
    operators."""
    shape = (1, 45, 70)
    cr = [dict(kind=1, eps=0.04, q=4, phi0=0.0)]
    seeds = [(30.0, 22.0, 0, 6.0, 0)]
    o = oracle_run(O, 0, shape, P2, cr, seeds=seeds, grad=grad, adv=V2)
    s = gpu_run(L, 0, shape, P2, cr, seeds=seeds, grad=grad, adv=V2)
    compare_chunks(o, s, (5, 48, 47), 1e-10)
    og, of = o.populations()
    assert maxabs(s.populations(1), of) <= 1e-12


@pytest.mark.parametrize("case", ["3d-z-walls", "3d-xy-walls", "2d-y-walls"])
def test_fp64_advection_along_walls(L, O, case):
    """Velocity tangential to the walls: the mirror image of the flow is the
    flow itself, so the bounce-back stays exact."""
    if case == "3d-z-walls":
        lat, shape, bc, v, prm = 1, (15, 20, 33), 4, (V3[0], V3[1], 0.0), P3
        cr, seeds = [dict(kind=0, eps=0.04)], [(12.0, 9.0, 0.0, 6.0, 0)]
    elif case == "3d-xy-walls":
        lat, shape, bc, v, prm = 1, (24, 17, 21), 3, (0.0, 0.0, V3[2] * 2), P3
        cr, seeds = [dict(kind=3, eps=0.0, gamma=-0.02)], [(0.0, 0.0, 12.0, 6.0, 0)]
    else:
        lat, shape, bc, v, prm = 0, (1, 40, 52), 2, V2[:1] + (0.0, 0.0), P2
        cr, seeds = [dict(kind=1, eps=0.04, q=6, phi0=0.1)], [(20.0, 0.0, 0, 7.0, 0)]
    o = oracle_run(O, lat, shape, prm, cr, seeds=seeds, bc=bc, adv=v)
    s = gpu_run(L, lat, shape, prm, cr, seeds=seeds, bc=bc, adv=v)
    compare_chunks(o, s, (9, 60), 1e-10)


def test_fp64_batched_with_and_without_flow(L, O):
    """One launch per step over two domains, one with a velocity and one
    without; each against its own oracle run."""
    specs = [((1, 45, 70), V2, [(30.0, 22.0, 0, 6.0, 0)]), ((1, 37, 52), (0.0, 0.0, 0.0), [(26.0, 18.0, 0, 5.0, 0)])]
    prm = dict(P2)
    lam = prm.pop("lam")
    cr = [dict(kind=1, eps=0.04, q=4, phi0=0.0)]
    doms, oracles = [], []
    for shape, v, seeds in specs:
        doms.append(L.make_domain(shape[2], shape[1], 1, lam=lam, crystals=[L.make_crystal(**c) for c in cr],
                                  adv=v, **prm))
        oracles.append(oracle_run(O, 0, shape, dict(prm, lam=lam), cr, seeds=seeds, adv=v))
    s = L.Solver(doms, 0, 0, L.LBPF_FP64)
    for k, (_, _, seeds) in enumerate(specs):
        s.seed(seeds, domain=k)
    for n in (40, 41):
        s.step(n)
        for k, o in enumerate(oracles):
            o.step(n)
            ophi, ou, _ = o.fields()
            assert maxabs(s.field(0, domain=k), ophi) <= 1e-10, (n, k)
            assert maxabs(s.field(1, domain=k), ou) <= 1e-10, (n, k)


def test_fp32_advective_growth(L, O):
    """FP32 full storage on a 40^3 periodic box through 300 steps: 1e-4 on
    phi and u at every checkpoint."""
    shape = (40, 40, 40)
    cr = [dict(kind=3, eps=0.0, gamma=-0.02)]
    seeds = [(20.0, 20.0, 20.0, 8.0, 0)]
    o = oracle_run(O, 1, shape, P3, cr, seeds=seeds, adv=V3)
    s = gpu_run(L, 1, shape, P3, cr, seeds=seeds, precision=L.LBPF_FP32, adv=V3)
    e = compare_chunks(o, s, (100, 100, 100), 1e-4)
    print(f"FP32 advective growth after 300 steps: phi {e[0]:.2e}, u {e[1]:.2e}")


def test_flow_breaks_the_symmetry(L):
    """A crystal in a flow along +x grows differently upstream and downstream
    (the upstream side sees fresh undercooled liquid): the tips along -x and
    +x differ, while the periodic run without flow keeps them equal."""
    shape = (40, 40, 64)
    cr = [dict(kind=0, eps=0.04)]
    seeds = [(32.0, 20.0, 20.0, 7.0, 0)]
    tips = {}
    for v in (0.0, 60.0):
        s = gpu_run(L, 1, shape, P3, cr, seeds=seeds, adv=(v, 0.0, 0.0))
        s.step(400)
        tips[v] = s.measure(32, 20, 20)[0]
        s.close()
    t0, t1 = tips[0.0], tips[60.0]
    assert abs(t0[0] - t0[1]) <= 1e-9
    # upstream (-x) against downstream (+x): the upstream tip is the longer
    # (the FP64 oracle: 29.0 against 8.4 sites, 14.4 both without flow)
    assert t1[1] - t1[0] > 5.0 and t1[1] > t0[1] > t1[0], (t0, t1)


@pytest.mark.parametrize("precision,bar", [(2, 1e-4), (3, 1e-3), (4, 1e-3)])
def test_dev16_advective_growth(L, O, precision, bar):
    """16-bit deviation storage (FP16, BF16, FP16 with stochastic rounding)
    with a flow: the stored heat deviations now carry w_j u (e_j . a), and the
    pull adds w_j (e_j . a) U as in full storage.  Against the FP64 oracle on
    a 40^3 periodic box through 300 steps (FP16 within 1e-4, BF16 and
    stochastic rounding within 1e-3 on phi and u), and Sum(u - phi/2), which
    advection conserves, to 1e-5 of its value."""
    shape = (40, 40, 40)
    cr = [dict(kind=3, eps=0.0, gamma=-0.02)]
    seeds = [(20.0, 20.0, 20.0, 8.0, 0)]
    o = oracle_run(O, 1, shape, P3, cr, seeds=seeds, adv=V3)
    s = gpu_run(L, 1, shape, P3, cr, seeds=seeds, precision=precision, adv=V3)
    c0 = s.measure(20, 20, 20)[2]
    e = compare_chunks(o, s, (100, 100, 100), bar)
    c1 = s.measure(20, 20, 20)[2]
    print(f"precision {precision}, advective growth after 300 steps: phi {e[0]:.2e}, u {e[1]:.2e}, "
          f"conserved drift {abs(c1 - c0) / abs(c0):.2e}")
    assert abs(c1 - c0) <= 1e-5 * abs(c0)


def test_fp16_advection_along_walls(L, O):
    """FP16 deviations, walls on z, velocity in the x-y plane."""
    shape = (15, 20, 33)
    cr, seeds = [dict(kind=0, eps=0.04)], [(12.0, 9.0, 0.0, 6.0, 0)]
    v = (V3[0], V3[1], 0.0)
    o = oracle_run(O, 1, shape, P3, cr, seeds=seeds, bc=4, adv=v)
    s = gpu_run(L, 1, shape, P3, cr, seeds=seeds, bc=4, adv=v, precision=2)
    e = compare_chunks(o, s, (9, 60), 1e-4)
    print(f"FP16 deviations, z walls, flow in x-y: phi {e[0]:.2e}, u {e[1]:.2e}")
