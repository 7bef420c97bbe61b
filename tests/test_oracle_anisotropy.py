"""Pins of the oracle's anisotropy functions and vector N (Secs. 2 and 4.1).

* Sec. 4.1: in 2D, 1 + eps cos(4 varphi) is the same function as
  1 - 3 eps + 4 eps (nx^4 + ny^4), and Eq. (As_Y66) is 1 + eps cos(6 varphi)
  in the XY plane: the polynomial forms and the angle form Eq. (As_Theta) are
  independent code paths, so equal a_s AND equal N pin both.
* Eq. (As_MatSci) is K00 + eps K41 + gamma K61 with cubic harmonics, which
  average to zero over the sphere and are mutually orthogonal: the sphere mean
  of a_s is exactly 1 and the constants 3/5 and 17/7 are fixed by that.
* Sec. 4.1 / Fig. 3: eps = 0, gamma = -0.02 favours <110>; the S form favours
  <111>; Eq. (As_Function_Classical) favours <100>.
* N of Eq. (TermesAnisotropes) is |grad phi|^2 a_s d a_s / d(grad phi):
  checked against central differences of a_s(grad phi); G . N = 0 because a_s
  depends on the direction of grad phi only; N commutes with the cube group.
"""
import numpy as np
import pytest


def a_of(O, cr, D, G):
    return O.anisotropy(cr, D, G)[0]


def unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


def test_cubic_equals_cos4_in_2d(orc):
    O = orc
    eps = 0.07
    cub = O.make_crystal(O.AS_CUBIC100, eps=eps)
    ang = O.make_crystal(O.AS_ANGLE, eps=eps, q=4, phi0=0.0)
    for vphi in np.linspace(0.01, 2 * np.pi, 37):
        G = -2.3 * np.array([np.cos(vphi), np.sin(vphi), 0.0])  # n = -G/|G|
        a1, N1 = O.anisotropy(cub, 2, G)
        a2, N2 = O.anisotropy(ang, 2, G)
        assert abs(a1 - (1 + eps * np.cos(4 * vphi))) < 1e-14
        assert abs(a1 - a2) < 1e-14
        assert np.abs(N1 - N2).max() < 1e-13


def test_y66_equals_cos6(orc):
    O = orc
    eps = 0.05
    y66 = O.make_crystal(O.AS_Y66, eps=eps)
    ang = O.make_crystal(O.AS_ANGLE, eps=eps, q=6, phi0=0.0)
    for vphi in np.linspace(0.02, 2 * np.pi, 41):
        G = -0.7 * np.array([np.cos(vphi), np.sin(vphi), 0.0])
        a1, N1 = O.anisotropy(y66, 2, G)
        a2, N2 = O.anisotropy(ang, 2, G)
        a3, N3 = O.anisotropy(y66, 3, G)  # 3D form on the XY plane
        assert abs(a1 - (1 + eps * np.cos(6 * vphi))) < 1e-14
        assert abs(a1 - a2) < 1e-14 and abs(a1 - a3) < 1e-14
        assert np.abs(N1 - N2).max() < 1e-13 and np.abs(N1 - N3).max() < 1e-13


def test_angle_form_orientation_and_odd_q(orc):
    """a_s(varphi) peaks at varphi = varphi0 + 2 pi k / q; for odd q the
    quadrant-aware angle gives q distinct maxima."""
    O = orc
    for q, ph0 in ((5, 0.3), (4, np.pi / 4), (6, 0.1)):
        cr = O.make_crystal(O.AS_ANGLE, eps=0.04, q=q, phi0=ph0)
        vs = np.linspace(0, 2 * np.pi, 3600, endpoint=False)
        a = np.array([a_of(O, cr, 2, -np.array([np.cos(v), np.sin(v), 0])) for v in vs])
        peaks = vs[(a > np.roll(a, 1)) & (a >= np.roll(a, -1))]
        assert len(peaks) == q
        d = np.angle(np.exp(1j * q * (peaks - ph0)))
        assert np.abs(d).max() < 2 * np.pi * q / 3600


def sphere_quadrature(nt=24, nph=48):
    x, wx = np.polynomial.legendre.leggauss(nt)  # cos(theta)
    ph = np.arange(nph) * 2 * np.pi / nph
    ct, P = np.meshgrid(x, ph, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    n = np.stack([st * np.cos(P), st * np.sin(P), ct], -1).reshape(-1, 3)
    w = (wx[:, None] * np.ones(nph)[None, :]).reshape(-1) * (2 * np.pi / nph) / (4 * np.pi)
    return n, w


def test_cubic_harmonics_mean_and_orthogonality(orc):
    O = orc
    n, w = sphere_quadrature()
    def mean_a(cr):
        return sum(wi * a_of(O, cr, 3, -ni) for ni, wi in zip(n, w))
    for eps, gam in ((0.05, 0.0), (0.0, -0.02), (0.02, 0.02), (-0.02, 0.02)):
        assert abs(mean_a(O.make_crystal(O.AS_HOYT110, eps=eps, gamma=gam)) - 1.0) < 1e-13
    # K41 and K61 parts are orthogonal on the sphere
    k41 = np.array([a_of(O, O.make_crystal(O.AS_HOYT110, eps=1.0), 3, -ni) - 1 for ni in n])
    k61 = np.array([a_of(O, O.make_crystal(O.AS_HOYT110, gamma=1.0), 3, -ni) - 1 for ni in n])
    assert abs((w * k41 * k61).sum()) < 1e-13
    assert (w * k41 * k41).sum() > 1e-3 and (w * k61 * k61).sum() > 1e-3


def test_preferred_directions(orc):
    O = orc
    dirs = {"100": unit([1, 0, 0]), "110": unit([1, 1, 0]), "111": unit([1, 1, 1])}
    def best(cr):
        vals = {k: a_of(O, cr, 3, -v) for k, v in dirs.items()}
        return max(vals, key=vals.get), vals
    assert best(O.make_crystal(O.AS_CUBIC100, eps=0.05))[0] == "100"
    assert best(O.make_crystal(O.AS_HOYT110, eps=0.0, gamma=-0.02))[0] == "110"
    assert best(O.make_crystal(O.AS_S111, gamma=0.02))[0] == "111"
    # the <111> form is 1 on the axes and 1 + 66 gamma / 27 on <111>
    v = best(O.make_crystal(O.AS_S111, gamma=0.02))[1]
    assert abs(v["100"] - 1) < 1e-15 and abs(v["111"] - (1 + 66 * 0.02 / 27)) < 1e-15
    # over a dense set of directions the maximum of the <110> form sits on <110>
    n, _ = sphere_quadrature(60, 120)
    cr = O.make_crystal(O.AS_HOYT110, eps=0.0, gamma=-0.02)
    a = np.array([a_of(O, cr, 3, -ni) for ni in n])
    nm = np.sort(np.abs(n[np.argmax(a)]))
    assert np.allclose(nm, [0, 1 / np.sqrt(2), 1 / np.sqrt(2)], atol=0.06)


KINDS = [("cubic", 2, dict(kind=0, eps=0.05)), ("cubic", 3, dict(kind=0, eps=0.05)),
         ("angle5", 2, dict(kind=1, eps=0.04, q=5, phi0=0.3)),
         ("y66", 2, dict(kind=2, eps=0.05)), ("y66", 3, dict(kind=2, eps=0.05)),
         ("hoyt", 3, dict(kind=3, eps=0.02, gamma=-0.02)), ("hoyt2d", 2, dict(kind=3, eps=0.02, gamma=-0.02)),
         ("s111", 3, dict(kind=4, gamma=0.02))]


@pytest.mark.parametrize("name,D,kw", KINDS)
def test_N_is_derivative_of_a(orc, name, D, kw):
    O = orc
    cr = O.make_crystal(**kw)
    rng = np.random.default_rng(7)
    for _ in range(20):
        G = rng.normal(size=3) * rng.uniform(0.1, 3)
        if D == 2:
            G[2] = 0
        a, N = O.anisotropy(cr, D, G)
        g2 = G @ G
        h = 1e-3 * np.sqrt(g2)
        dadG = np.zeros(3)
        for al in range(D):
            e = np.zeros(3)
            e[al] = h
            # fourth-order central difference
            dadG[al] = (8 * (a_of(O, cr, D, G + e) - a_of(O, cr, D, G - e))
                        - (a_of(O, cr, D, G + 2 * e) - a_of(O, cr, D, G - 2 * e))) / (12 * h)
        Nfd = g2 * a * dadG
        strength = abs(kw.get("eps", 0)) + abs(kw.get("gamma", 0))
        assert np.abs(N - Nfd).max() <= 1e-8 * strength * np.sqrt(g2), (N, Nfd)
        assert abs(G @ N) <= 1e-13 * np.sqrt(g2) * max(1e-12, np.abs(N).max()) * 10


def signed_perms():
    from itertools import permutations, product
    for p in permutations(range(3)):
        for s in product((1, -1), repeat=3):
            P = np.zeros((3, 3))
            for i in range(3):
                P[i, p[i]] = s[i]
            yield P


@pytest.mark.parametrize("kw", [dict(kind=0, eps=0.05), dict(kind=3, eps=0.02, gamma=-0.02), dict(kind=4, gamma=0.02)])
def test_cubic_group_covariance(orc, kw):
    O = orc
    cr = O.make_crystal(**kw)
    G = np.array([0.3, -1.1, 0.7])
    a0, N0 = O.anisotropy(cr, 3, G)
    for P in signed_perms():
        a, N = O.anisotropy(cr, 3, P @ G)
        assert abs(a - a0) < 1e-14 and np.abs(N - P @ N0).max() < 1e-14


def test_zero_gradient_guard(orc):
    O = orc
    a, N = O.anisotropy(O.make_crystal(O.AS_CUBIC100, eps=0.05), 3, [0, 0, 0])
    assert a == 1.0 and not N.any()
