"""Pins of the oracle's gradient operators (Sec. 4.2).

Directional derivatives, Eq. (Def_DeriveeDirectionnelle) + Eq.
(Grad_DF-Centree), and central finite differences are checked against what
Taylor series and lattice isotropy fix exactly:
  * on any polynomial of degree <= 4, DD = grad(phi) + (dx^2/6) grad(lap phi)
    on a fourth-order isotropic lattice, and FD_a = d_a phi + (dx^2/6) d_a^3 phi;
  * on a periodic Fourier mode, DD = (1/e^2) sum_i w_i e_i sin(k.e_i dx)/dx
    times the phase-shifted mode (exercises the periodic wrap as well);
  * the isotropy contrast the paper claims: on a tanh sphere the DD gradient
    direction converges faster to the radial direction than the FD one.
"""
from itertools import product

import numpy as np
import pytest


def monomials(D, deg=4):
    return [m for m in product(range(deg + 1), repeat=3) if sum(m) <= deg and (D == 3 or m[2] == 0)]


def deriv(poly, axis, order=1):
    out = {}
    for m, c in poly.items():
        k = m[axis]
        if k < order:
            continue
        f = 1
        for j in range(order):
            f *= k - j
        mm = list(m)
        mm[axis] -= order
        out[tuple(mm)] = out.get(tuple(mm), 0.0) + c * f
    return out


def add(*ps):
    out = {}
    for p in ps:
        for m, c in p.items():
            out[m] = out.get(m, 0.0) + c
    return out


def evaluate(poly, X, Y, Z):
    v = np.zeros_like(X)
    for (a, b, c), co in poly.items():
        v += co * X ** a * Y ** b * Z ** c
    return v


@pytest.mark.parametrize("lat", [0, 1, 2, 3])
@pytest.mark.parametrize("grad", [0, 1])
def test_polynomial_exactness(orc, lat, grad):
    O = orc
    D = O.lattice(lat, 0)[0]
    rng = np.random.default_rng(100 + 10 * lat + grad)
    poly = {m: rng.uniform(-1, 1) for m in monomials(D)}
    n = 12
    nz = n if D == 3 else 1
    dx = 0.25
    p = O.make_params(lat, n, n, nz, grad=grad, dx=dx)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(n), np.arange(n), indexing="ij")
    X, Y, Z = x * dx, y * dx, z * dx
    G = O.gradient(p, evaluate(poly, X, Y, Z))
    lap = add(*[deriv(deriv(poly, a), a) for a in range(D)])
    sl = (slice(1, -1) if D == 3 else slice(None), slice(1, -1), slice(1, -1))
    scale = max(np.abs(evaluate(deriv(poly, a), X, Y, Z)[sl]).max() for a in range(D))
    for a in range(D):
        if grad == 0:
            want = evaluate(add(deriv(poly, a), {m: c * dx * dx / 6 for m, c in deriv(lap, a).items()}), X, Y, Z)
        else:
            want = evaluate(add(deriv(poly, a), {m: c * dx * dx / 6 for m, c in deriv(poly, a, 3).items()}), X, Y, Z)
        err = np.abs(G[..., a][sl] - want[sl]).max()
        assert err <= 1e-12 * scale, (a, err, scale)
    if D == 2:
        assert np.all(G[..., 2] == 0)


@pytest.mark.parametrize("lat", [0, 1, 2, 3])
def test_fourier_mode_dd(orc, lat):
    O = orc
    D, e, w, e2 = O.lattice(lat, 0)
    nx, ny, nz = 16, 12, (10 if D == 3 else 1)
    dx = 0.3
    m = np.array([3, -2, 1 if D == 3 else 0])
    k = 2 * np.pi * m / (np.array([nx, ny, nz]) * dx)
    p = O.make_params(lat, nx, ny, nz, grad=0, dx=dx)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    th = k[0] * x * dx + k[1] * y * dx + k[2] * z * dx + 0.4
    G = O.gradient(p, np.sin(th))
    amp = sum(wi * ei * np.sin(dx * (k @ ei)) for ei, wi in zip(e, w)) / (e2 * dx)
    for a in range(3):
        assert np.abs(G[..., a] - amp[a] * np.cos(th)).max() < 1e-12


def angular_error(O, lat, grad, W):
    """Max angle (rad) between the numerical gradient of a tanh sphere of width
    W (lattice units) and the radial direction, over the interface shell."""
    n = 40
    p = O.make_params(lat, n, n, n, grad=grad, dx=1.0)
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    c = n / 2 + 0.37
    r = np.sqrt((x - c) ** 2 + (y - c - 0.21) ** 2 + (z - c + 0.13) ** 2)
    R = 10.0
    G = O.gradient(p, np.tanh((R - r) / W))
    shell = np.abs(r - R) < 1.0
    rad = -np.stack([x - c, y - c - 0.21, z - c + 0.13], -1) / r[..., None]
    cosang = (G * rad).sum(-1) / np.linalg.norm(G, axis=-1)
    return np.arccos(np.clip(cosang[shell], -1, 1)).max()


def test_dd_more_isotropic_than_fd(orc):
    """Sec. 4.2 claims DD reduces lattice anisotropy of the gradient.  On a
    sphere both errors shrink with the interface width; DD's anisotropic part
    is O(dx^4) (the dx^2 term is isotropic, grad(lap phi) of a radial field
    is radial), FD's is O(dx^2)."""
    O = orc
    for W in (2.0, 4.0):
        dd = angular_error(O, O.D3Q15_D3Q7, 0, W)
        fd = angular_error(O, O.D3Q15_D3Q7, 1, W)
        assert dd < 0.25 * fd, (W, dd, fd)
    r_dd = angular_error(O, O.D3Q15_D3Q7, 0, 2.0) / angular_error(O, O.D3Q15_D3Q7, 0, 4.0)
    r_fd = angular_error(O, O.D3Q15_D3Q7, 1, 2.0) / angular_error(O, O.D3Q15_D3Q7, 1, 4.0)
    assert r_dd > 8.0 and 2.5 < r_fd < 6.0, (r_dd, r_fd)
