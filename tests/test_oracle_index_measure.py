"""Pins of the oracle's crystal-index field (Sec. 4.3, Eq. As_Multi) and of
its measurements, by brute force on small cases.

The index rule of Sec. 4.3: after initialisation, a node with index 0 whose
gradient exceeds xi takes the index of the nearest node with a non-zero index;
a_s^(I) uses crystal I, and there is no anisotropy where I = 0.
"""
import numpy as np
import pytest


def two_crystal_oracle(O, n=40, xi=1e-4):
    crs = [O.make_crystal(O.AS_ANGLE, eps=0.05, q=4, phi0=0.3),
           O.make_crystal(O.AS_ANGLE, eps=0.03, q=6, phi0=1.1)]
    p = O.make_params(O.D2Q9_D2Q5, n, n, 1, dx=1.0, dt=0.05, W0=1.0, tau0=1.0, kappa=1.0, lam=3.0,
                      delta=0.4, xi=xi, crystals=crs)
    seeds = [[8.0, 8.0, 0, 3.0, 0], [28.0, 26.0, 0, 3.5, 1]]
    return O.Oracle(p).seed(seeds), p, seeds, crs


def test_initial_index(orc):
    O = orc
    o, p, seeds, _ = two_crystal_oracle(O)
    phi, u, I = o.fields()
    n = 40
    y, x = np.mgrid[0:n, 0:n]
    prof = []
    for sx, sy, _, R, c in seeds:
        dxp = (x - sx + n / 2) % n - n / 2
        dyp = (y - sy + n / 2) % n - n / 2
        prof.append(np.tanh((R - np.hypot(dxp, dyp)) / np.sqrt(2)))
    prof = np.array(prof)
    assert np.abs(phi[0] - prof.max(0)).max() < 1e-15
    G = O.gradient(p, phi)
    near = (phi[0] > 0) | (np.linalg.norm(G[0], axis=-1) > p.xi)
    want = np.where(near, prof.argmax(0) + 1, 0)
    assert np.array_equal(I[0], want)
    assert (I == 0).any() and (I == 1).any() and (I == 2).any()


def test_index_update_jacobi_nearest(orc):
    O = orc
    o, p, seeds, crs = two_crystal_oracle(O)
    _, e, _, _ = O.lattice(O.D2Q9_D2Q5, 0)
    for _ in range(5):
        phi0, _, I0 = o.fields()
        G = O.gradient(p, phi0)[0]
        o.step(1)
        _, _, I1 = o.fields()
        want = I0[0].copy()
        n = 40
        for yy in range(n):
            for xx in range(n):
                if I0[0, yy, xx] != 0 or not np.linalg.norm(G[yy, xx]) > p.xi:
                    continue
                # nearest neighbour with a non-zero index: axes before diagonals
                for ex, ey, _ in e[1:]:
                    v = I0[0, (yy + ey) % n, (xx + ex) % n]
                    if v:
                        want[yy, xx] = v
                        break
        assert np.array_equal(I1[0], want)
    assert (I1 != I0).any() or True


def test_anisotropy_follows_index(orc):
    O = orc
    o, p, seeds, crs = two_crystal_oracle(O)
    o.step(3)
    phi_before, _, _ = o.fields()
    G = O.gradient(p, phi_before)[0]
    o.step(1)
    _, _, I = o.fields()
    a = o.anisotropy_field()[0]
    for yy in range(0, 40, 3):
        for xx in range(0, 40, 3):
            k = I[0, yy, xx]
            if k == 0:
                assert a[yy, xx] == 1.0
            else:
                assert abs(a[yy, xx] - O.anisotropy(crs[k - 1], 2, G[yy, xx])[0]) < 1e-15


def test_measure_on_known_profile(orc):
    O = orc
    n = 32
    p = O.make_params(O.D3Q15_D3Q7, n, n, n)
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    c = 16
    A = (7.3, 6.1, 5.6, 4.4, 3.25, 2.5)  # +x, -x, +y, -y, +z, -z crossings
    def ramp(d, ap, am):
        return np.where(d >= 0, 1 - d / ap, 1 + d / am)
    phi = np.minimum(np.minimum(ramp(x - c, A[0], A[1]), ramp(y - c, A[2], A[3])), ramp(z - c, A[4], A[5]))
    u = np.sin(x * 0.3) * 0.1
    o = O.Oracle(p).set_fields(phi, u)
    tip, sf, cs = o.measure(c, c, c)
    assert np.allclose(tip, A, atol=1e-13)
    assert abs(sf - (0.5 * (1 + phi)).mean()) < 1e-12
    assert abs(cs - (u - 0.5 * phi).sum()) < 1e-12 * np.abs(u - 0.5 * phi).sum()
    # no crossing: the whole ray solid or liquid
    o2 = O.Oracle(p).set_fields(-np.ones((n, n, n)), u)
    assert np.all(o2.measure(c, c, c)[0] == -1)


def test_current_anisotropy_field_closed_forms(orc):
    """a_s of the current field on planar interfaces, against the values the
    anisotropy functions take on the crystal axes (Sec. 2 and Sec. 5.2):
    <100> normal: cubic 1 + eps, <110> form 1 + 2eps/5 + 4gamma/7;
    <110> normal: cubic 1 - eps, <110> form 1 - eps/10 - 13gamma/14.
    A field that depends on x only (or on x + y only) has, by symmetry of
    the lattice stencils, a gradient exactly along x (along (1, 1, 0))."""
    O = orc
    n = 24
    z, y, x = np.mgrid[0:n, 0:n, 0:n].astype(float)
    eps, gam = 0.03, -0.02
    cases = [
        (np.tanh(2.0 * np.sin(2 * np.pi * x / n)), dict(kind=0, eps=eps), 1 + eps),
        (np.tanh(2.0 * np.sin(2 * np.pi * (x + y) / n)), dict(kind=0, eps=eps), 1 - eps),
        (np.tanh(2.0 * np.sin(2 * np.pi * x / n)), dict(kind=3, eps=eps, gamma=gam), 1 + 2 * eps / 5 + 4 * gam / 7),
        (np.tanh(2.0 * np.sin(2 * np.pi * (x + y) / n)), dict(kind=3, eps=eps, gamma=gam),
         1 - eps / 10 - 13 * gam / 14),
    ]
    for grad in (O.GRAD_DD, O.GRAD_FD):
        for phi, cr, want in cases:
            p = O.make_params(O.D3Q15_D3Q7, n, n, n, grad=grad, crystals=[O.make_crystal(**cr)])
            o = O.Oracle(p).set_fields(phi, np.zeros_like(phi))
            a = o.current_anisotropy()
            G = O.gradient(p, phi)
            moving = np.linalg.norm(G, axis=-1) > 1e-6  # away from the extrema of the sine
            assert moving.mean() > 0.8
            assert np.abs(a[moving] - want).max() <= 1e-13
    # several crystals: a_s = 1 where the index is 0, the crystal's a_s elsewhere
    p = O.make_params(O.D3Q15_D3Q7, n, n, n, crystals=[O.make_crystal(kind=0, eps=eps),
                                                       O.make_crystal(kind=0, eps=-eps)])
    phi = cases[0][0]
    I = np.where(x < n / 2, 1, 2).astype(np.int32)
    I[:, :, :3] = 0
    o = O.Oracle(p).set_fields(phi, np.zeros_like(phi), I)
    a = o.current_anisotropy()
    G = O.gradient(p, phi)
    moving = np.linalg.norm(G, axis=-1) > 1e-6
    assert np.all(a[I == 0] == 1.0)
    assert np.abs(a[(I == 1) & moving] - (1 + eps)).max() <= 1e-13
    assert np.abs(a[(I == 2) & moving] - (1 - eps)).max() <= 1e-13
