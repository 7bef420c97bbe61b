"""Pins of the oracle's zero-flux walls (Sec. 3.3) and of the octant runs of
Sec. 5.3.

A wall is a mirror plane through the boundary nodes.  A box of n nodes with
walls at both ends of an axis is then exactly a part of the periodic run of
period 2(n - 1) whose initial state is mirror-symmetric about nodes 0 and
n - 1: the periodic scheme (pinned separately) keeps that symmetry, and the
walls must reproduce it node for node, to rounding.  This pins every wall
ingredient at once: the gradient stencil and the non-local term of Eq.
(LBE_Eq_Phase) at the wall, the reflected populations after streaming, and
the index field near walls.  The seeds of the octant run of Sec. 5.3 sit at
the origin, on three walls.
"""
import numpy as np
import pytest

P3 = dict(dx=0.01, dt=1.5e-5, W0=0.0125, tau0=1.5625e-4, kappa=1.0, lam=10.0, delta=0.25)
P2 = dict(dx=0.4, dt=0.008, W0=1.0, tau0=1.0, kappa=2.0, delta=0.3)


def mirror_extend(a, axes):
    """The mirror-symmetric periodic extension (period 2(n-1)) of a field
    given on n nodes, along the given array axes."""
    for ax in axes:
        n = a.shape[ax]
        inner = np.flip(np.take(a, np.arange(1, n - 1), axis=ax), axis=ax)
        a = np.concatenate([a, inner], axis=ax)
    return a


def images(seeds, box, walls):
    """Seeds and their mirror images across the walled axes (x, y, z)."""
    out = []
    for s in seeds:
        cands = [list(s)]
        for a in range(3):
            if walls >> a & 1:
                cands = cands + [c[:a] + [-c[a]] + c[a + 1:] for c in cands]
        out += cands
    return out


def run_pair(O, lattice, box, walls, crystals, prm, steps, seeds=None, fields=None, grad=0):
    """(wall run, periodic mirror run restricted to the box) after steps."""
    nz, ny, nx = box
    D = 2 if lattice == 0 else 3
    axes_arr = [2 - a for a in range(D) if walls >> a & 1]  # array axes of the walled x, y, z
    big = list(box)
    for ax in axes_arr:
        big[ax] = 2 * (box[ax] - 1)
    crs = [O.make_crystal(**c) for c in crystals]
    pw = O.make_params(lattice, nx, ny, nz, grad=grad, crystals=crs, bc=walls, **prm)
    pp = O.make_params(lattice, big[2], big[1], big[0], grad=grad, crystals=crs, **prm)
    ow, op = O.Oracle(pw), O.Oracle(pp)
    if seeds is not None:
        ow.seed(seeds)
        op.seed(images(seeds, box, walls))
    else:
        phi, u = fields
        ow.set_fields(phi, u)
        op.set_fields(mirror_extend(phi, axes_arr), mirror_extend(u, axes_arr))
    ow.step(steps)
    op.step(steps)
    sl = tuple(slice(0, n) for n in box)
    wf, pf = ow.fields(), op.fields()
    return ow, op, wf, tuple(f[sl] for f in pf)


@pytest.mark.parametrize("lattice", [1, 2, 3])
@pytest.mark.parametrize("form", [dict(kind=0, eps=0.05), dict(kind=3, eps=0.0, gamma=-0.02)])
def test_octant_equals_mirror_symmetric_run(orc, lattice, form):
    """The octant of Sec. 5.3: seed at the origin, walls on all six faces."""
    box = (10, 11, 12)
    ow, op, (phi, u, I), (pphi, pu, pI) = run_pair(orc, lattice, box, 7, [form], P3, 60,
                                                   seeds=[(0.0, 0.0, 0.0, 6.0, 0)])
    assert np.abs(phi - pphi).max() <= 1e-13 and np.abs(u - pu).max() <= 1e-13
    assert np.abs(phi - phi[0, 0, 0]).max() > 0.5  # an interface crosses the box


@pytest.mark.parametrize("grad", [0, 1])
def test_closed_box_random_fields(orc, grad):
    """Arbitrary (not symmetric) fields in a closed box: every wall node
    differs from its neighbours, so the reflected populations, the gradient
    and the non-local term at walls, edges and corners are all exercised."""
    rng = np.random.default_rng(11)
    box = (9, 10, 13)
    z, y, x = np.mgrid[0:9, 0:10, 0:13]
    phi = np.tanh(1.5 * np.sin(0.7 * x + 0.3) * np.cos(0.5 * y - 0.2) + 0.4 * np.sin(0.9 * z) +
                  0.1 * rng.standard_normal(box))
    u = -0.3 + 0.05 * rng.standard_normal(box)
    ow, op, (wphi, wu, _), (pphi, pu, _) = run_pair(orc, 1, box, 7, [dict(kind=3, eps=0.02, gamma=-0.02)], P3, 40,
                                                    fields=(phi, u), grad=grad)
    assert np.abs(wphi - pphi).max() <= 1e-13 and np.abs(wu - pu).max() <= 1e-13


def test_mixed_walls_and_2d(orc):
    """Walls along x only (y, z periodic) in 3D; walls along y only in 2D
    (fourfold angle form with phi0 = 0, symmetric under both reflections)."""
    rng = np.random.default_rng(3)
    box = (8, 9, 12)
    phi = np.tanh(rng.standard_normal(box))
    u = -0.2 + 0.02 * rng.standard_normal(box)
    _, _, (a, b, _), (c, d, _) = run_pair(orc, 1, box, 1, [dict(kind=0, eps=0.04)], P3, 30, fields=(phi, u))
    assert np.abs(a - c).max() <= 1e-13 and np.abs(b - d).max() <= 1e-13
    box2 = (1, 15, 20)
    seeds = [(4.0, 0.0, 0.0, 5.0, 0), (13.0, 9.0, 0.0, 4.0, 0)]
    _, _, (a, b, _), (c, d, _) = run_pair(orc, 0, box2, 2, [dict(kind=1, eps=0.05, q=4, phi0=0.0)], P2, 200,
                                          seeds=seeds)
    assert np.abs(a - c).max() <= 1e-12 and np.abs(b - d).max() <= 1e-12


def test_index_field_at_walls(orc):
    """Three crystals near walls (2D, walls on both axes): the index field of
    the wall run equals the mirror-symmetric periodic run's."""
    box = (1, 24, 28)
    prm = dict(dx=5e-3, dt=5e-6, W0=0.012, tau0=1e-4, kappa=0.7, lam=10.0, delta=0.35)
    crs = [dict(kind=1, eps=0.04, q=4, phi0=0.0), dict(kind=1, eps=0.04, q=4, phi0=np.pi / 4),
           dict(kind=1, eps=0.03, q=4, phi0=0.0)]
    seeds = [(0.0, 0.0, 0.0, 4.0, 0), (20.0, 3.0, 0.0, 4.5, 1), (9.0, 22.0, 0.0, 4.0, 2)]
    O = orc
    ow, op, (phi, u, I), (pphi, pu, pI) = run_pair(O, 0, box, 3, crs, prm, 150, seeds=seeds)
    assert np.array_equal(I, pI)
    assert np.abs(phi - pphi).max() <= 1e-12 and set(np.unique(I)) >= {0, 1, 2, 3}


def test_closed_box_conservation(orc):
    """Zero flux through the walls: the trapezoid-weighted sum of u - phi/2
    (nodes on the mirror planes count 1/2 per walled coordinate) is constant
    to rounding; without the weights it drifts."""
    O = orc
    rng = np.random.default_rng(7)
    box = (10, 11, 12)
    phi = np.tanh(2.0 * rng.standard_normal(box))
    u = -0.3 + 0.1 * rng.standard_normal(box)
    p = O.make_params(1, 12, 11, 10, crystals=[O.make_crystal(kind=0, eps=0.05)], bc=7, **P3)
    o = O.Oracle(p).set_fields(phi, u)
    c0 = o.measure(0, 0, 0)[2]
    o.step(300)
    c1 = o.measure(0, 0, 0)[2]
    ph, uu, _ = o.fields()
    assert abs(c1 - c0) <= 1e-12 * np.abs(u - 0.5 * phi).sum()
    plain0 = (u - 0.5 * phi).sum()
    plain1 = (uu - 0.5 * ph).sum()
    assert abs(plain1 - plain0) > 1e-6  # the unweighted sum is not the invariant


def test_tips_stop_at_walls(orc):
    """Tip rays from the octant's origin run to the far wall, and the tip
    equals the one of the mirror-symmetric periodic run (half its period)."""
    O = orc
    box = (12, 12, 12)
    ow, op, (phi, _, _), _ = run_pair(O, 1, box, 7, [dict(kind=0, eps=0.05)], P3, 100,
                                      seeds=[(0.0, 0.0, 0.0, 7.0, 0)])
    tw = ow.measure(0, 0, 0)[0]
    tp = op.measure(0, 0, 0)[0]
    assert np.allclose(tw[[0, 2, 4]], tp[[0, 2, 4]], atol=1e-12) and tw[0] > 7.0
    assert np.all(tw[[1, 3, 5]] == -1)  # nothing behind the origin inside the box
