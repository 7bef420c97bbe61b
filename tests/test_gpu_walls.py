"""Zero-flux walls (Sec. 3.3) on the GPU against the FP64 oracle.

Walls are mirror planes through the boundary nodes (include/lbpf.h,
LBPF_BC_WALL_X); the oracle's walls are pinned on the CPU by the equality of
an octant run with the mirror-symmetric periodic run.  Here the CUDA path
(through the C ABI) must match the oracle element by element: FP64 within
1e-10 on phi and u, FP32 within 1e-4 with tips within 0.5 lattice unit.
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


def random_fields(shape, seed):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    phi = np.tanh(1.5 * np.sin(0.7 * x + 0.3) * np.cos(0.5 * y - 0.2) + 0.4 * np.sin(0.9 * z) +
                  0.1 * rng.standard_normal(shape))
    u = -0.3 + 0.05 * rng.standard_normal(shape)
    return phi, u


@pytest.mark.parametrize("lattice", [1, 2, 3])
@pytest.mark.parametrize("grad", [0, 1])
def test_fp64_octant(L, O, lattice, grad):
    """Octant of Sec. 5.3 (seed at the origin, walls on all faces), ragged
    tiles in x and y; the state, the populations, the tips and the
    trapezoid-weighted conserved sum."""
    shape = (19, 22, 37)
    cr = [dict(kind=3, eps=0.0, gamma=-0.02)]
    seeds = [(0.0, 0.0, 0.0, 8.0, 0)]
    o = oracle_run(O, lattice, shape, P3, cr, seeds=seeds, grad=grad, bc=7)
    s = gpu_run(L, lattice, shape, P3, cr, seeds=seeds, grad=grad, bc=7)
    _, _, c0 = s.measure(0, 0, 0)
    o.step(120)
    s.step(120)
    phi, u = s.fields()
    ophi, ou, _ = o.fields()
    assert maxabs(phi, ophi) <= 1e-10 and maxabs(u, ou) <= 1e-10
    tip, _, c1 = s.measure(0, 0, 0)
    otip, _, oc = o.measure(0, 0, 0)
    assert np.abs(tip - otip).max() <= 1e-9 and abs(c1 - oc) <= 1e-9 * abs(oc)
    assert abs(c1 - c0) <= 1e-12 * abs(c0)
    assert tip[0] > 7.0 and np.all(tip[[1, 3, 5]] == -1)
    if lattice == 1:
        og, of = o.populations()
        assert maxabs(s.populations(0), og) <= 1e-12 and maxabs(s.populations(1), of) <= 1e-12


@pytest.mark.parametrize("bc", [1, 2, 4, 3, 7])
def test_fp64_closed_and_mixed_boxes(L, O, bc):
    """Arbitrary fields: every wall, edge and corner node differs from its
    neighbours.  Walls on some axes, periodic on the others."""
    shape = (11, 13, 40)
    phi, u = random_fields(shape, 5 + bc)
    cr = [dict(kind=0, eps=0.05)]
    o = oracle_run(O, 1, shape, P3, cr, fields=(phi, u), bc=bc)
    s = gpu_run(L, 1, shape, P3, cr, fields=(phi, u), bc=bc)
    o.step(50)
    s.step(50)
    p, uu = s.fields()
    assert maxabs(p, o.fields()[0]) <= 1e-10 and maxabs(uu, o.fields()[1]) <= 1e-10


@pytest.mark.parametrize("grad", [0, 1])
def test_fp64_2d_walls_multicrystal(L, O, grad):
    """2D, walls on both axes, three crystals (one on the corner), the index
    field at the paper's threshold xi = 1e-7 (Sec. 4.3)."""
    shape = (1, 50, 70)
    prm = dict(W.C4_PARAMS, delta=0.35)
    crs = [dict(kind=1, eps=0.04, q=4, phi0=0.0), dict(kind=1, eps=0.04, q=5, phi0=0.087),
           dict(kind=1, eps=0.04, q=6, phi0=0.3)]
    seeds = [(0.0, 0.0, 0, 6.0, 0), (50.0, 18.0, 0, 6.0, 1), (35.0, 45.0, 0, 4.5, 2)]
    o = oracle_run(O, 0, shape, prm, crs, seeds=seeds, grad=grad, xi=1e-7, bc=3)
    s = gpu_run(L, 0, shape, prm, crs, seeds=seeds, grad=grad, xi=1e-7, bc=3)
    for _ in range(3):
        o.step(100)
        s.step(100)
        ophi, ou, oI = o.fields()
        phi, u = s.fields()
        assert np.array_equal(s.field(L.LBPF_FIELD_INDEX), oI)
        assert maxabs(phi, ophi) <= 1e-10 and maxabs(u, ou) <= 1e-10
    tip, _, _ = s.measure(0, 0, 0)
    otip, _, _ = o.measure(0, 0, 0)
    assert np.abs(tip - otip).max() <= 1e-9
    for d in (0, 2):
        r = s.tip_radius(0, 0, 0, d, J=3)
        ro = O.tip_radius(ophi, (0, 0, 0), d, J=3, bc=3)
        assert abs(r - ro) <= 1e-8 * max(1.0, abs(ro)), (d, r, ro)


def test_fp32_octant_vs_oracle(L, O):
    """FP32 octant: 1e-4 on phi and u, tips within 0.5 lattice unit, at every
    checkpoint through 600 steps."""
    shape = (40, 40, 40)
    cr = [dict(kind=3, eps=0.0, gamma=-0.02)]
    seeds = [(0.0, 0.0, 0.0, 8.0, 0)]
    o = oracle_run(O, 1, shape, P3, cr, seeds=seeds, bc=7)
    s = gpu_run(L, 1, shape, P3, cr, seeds=seeds, precision=L.LBPF_FP32, bc=7)
    for k in range(3):
        o.step(200)
        s.step(200)
        phi, u = s.fields()
        ophi, ou, _ = o.fields()
        tip = s.measure(0, 0, 0)[0]
        otip = o.measure(0, 0, 0)[0]
        e = (maxabs(phi, ophi), maxabs(u, ou), np.abs(tip - otip).max())
        print(f"FP32 octant after {200 * (k + 1)} steps: phi {e[0]:.2e}, u {e[1]:.2e}, tips {e[2]:.2e}")
        assert e[0] <= 1e-4 and e[1] <= 1e-4 and e[2] <= 0.5


@pytest.mark.parametrize("precision", [2, 3])
def test_dev16_octant(L, O, precision):
    """16-bit deviation storage with walls: errors against the FP64 oracle are
    stated, with the sanity bounds of the periodic test; the weighted
    conserved sum holds to the storage's rounding."""
    shape = (40, 40, 40)
    cr = [dict(kind=3, eps=0.0, gamma=-0.02)]
    seeds = [(0.0, 0.0, 0.0, 8.0, 0)]
    o = oracle_run(O, 1, shape, P3, cr, seeds=seeds, bc=7)
    s = gpu_run(L, 1, shape, P3, cr, seeds=seeds, precision=precision, bc=7)
    _, _, c0 = s.measure(0, 0, 0)
    o.step(400)
    s.step(400)
    phi, u = s.fields()
    ophi, ou, _ = o.fields()
    tip, _, c1 = s.measure(0, 0, 0)
    otip = o.measure(0, 0, 0)[0]
    e = (maxabs(phi, ophi), maxabs(u, ou), np.abs(tip - otip).max(), abs(c1 - c0) / abs(c0))
    print(f"{'FP16' if precision == 2 else 'BF16'} deviations, octant, 400 steps: phi {e[0]:.2e}, u {e[1]:.2e}, "
          f"tips {e[2]:.2e}, drift {e[3]:.2e}")
    assert e[0] < 1.0 and e[1] < 0.5 and e[2] < 1.0 and e[3] <= 1e-5


def test_wall_arguments(L):
    d = L.make_domain(16, 16, 1, dx=1, dt=0.1, W0=1, tau0=1, kappa=1, bc=4)
    with pytest.raises(L.LbpfError):
        L.Solver(d, 0)  # no z wall in 2D
    d = L.make_domain(2, 16, 8, dx=1, dt=0.1, W0=1, tau0=1, kappa=1, bc=1)
    with pytest.raises(L.LbpfError):
        L.Solver(d, 1)  # a walled axis needs 3 sites
    d = L.make_domain(16, 16, 8, dx=1, dt=0.1, W0=1, tau0=1, kappa=1, bc=8)
    with pytest.raises(L.LbpfError):
        L.Solver(d, 1)
