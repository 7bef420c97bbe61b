"""Paper-scale runs of Younsi & Cartalade's isotropy experiments through the
library (every step on the GPU), with the quantities the paper reports.

Sec. 4.2 (Figs. 4-6): a sixfold 2D crystal (Eq. As_Theta, q = 6, phi0 = 0) on
800 x 800 nodes, grown for 10^5 steps with central finite differences (FD) or
directional derivatives (DD); the paper reports the relative l2 error of Eq.
(Error_L2) between the phi profiles along n_a = (1, 0) and n_b = (1/2,
-sqrt(3)/2) (FD 1.71e-1, DD 3.04e-3), and the extreme values of phi_rot -
phi, phi rotated by 60 degrees (FD 1.446 / -1.454, DD 0.1 / -0.103).

Sec. 5.2 (Figs. 7-8): dendrites A (<100>, Eq. As_Function_Classical, eps =
0.05, 5e3 steps), B (<110>, Eq. As_MatSci, eps = 0, gamma = -0.02, 2.5e4
steps) and C (<111>, Eq. As_Function_S, gamma = 0.02, 1.5e4 steps) on 351^3
nodes, Delta = 0.30, seed at the centre; the paper compares phi on two slices
through the centre after a rotation: A the planes of normals (1, 0, 0) and
(0, 1, 0), B (1, 1, 1) and (1, 1, -1), C (1, 1, 0) and (1, -1, 0).  Each pair
is related by a symmetry of the cube (a 90-degree rotation about z for A and
C, the reflection z -> -z for B), so a scheme on a cubic lattice reproduces
it to rounding; the differences reported here measure that.

The paper imposes zero fluxes on all boundaries (Sec. 2), so both runs use
walls on every face (include/lbpf.h, LBPF_BC_WALL_X).  Readings: the 3D seed
radius (not stated) is 8 sites; the profiles run from the centre to the
wall at unit spacing, sampled by bilinear interpolation; the 60-degree
rotation is compared on the disk that stays inside the domain.
"""
from __future__ import annotations

import math

import numpy as np

SEC42 = dict(dx=0.01, dt=1.5e-5, W0=0.0125, tau0=1.5625e-4, kappa=1.0, lam=10.0, delta=0.30)
SEC52 = dict(dx=0.01, dt=1.5e-5, W0=0.0125, tau0=1.5625e-4, kappa=1.0, lam=10.0, delta=0.30)
DENDRITES = {
    "A": (dict(kind=0, eps=0.05), 5000),
    "B": (dict(kind=3, eps=0.0, gamma=-0.02), 25000),
    "C": (dict(kind=4, gamma=0.02), 15000),
}


def bilinear(phi, ys, xs):
    """phi[y, x] at real positions (bilinear; positions inside the array)."""
    y0 = np.floor(ys).astype(int)
    x0 = np.floor(xs).astype(int)
    y1 = np.minimum(y0 + 1, phi.shape[0] - 1)
    x1 = np.minimum(x0 + 1, phi.shape[1] - 1)
    fy, fx = ys - y0, xs - x0
    return ((1 - fy) * ((1 - fx) * phi[y0, x0] + fx * phi[y0, x1]) +
            fy * ((1 - fx) * phi[y1, x0] + fx * phi[y1, x1]))


def err_l2(pa, pb):
    """Eq. (Error_L2), profile a taken as the reference."""
    return float(np.sqrt(((pa - pb) ** 2).sum() / (pa ** 2).sum()))


def isotropy_measures(phi, c):
    """Err_l2 of the profiles along n_a and n_b, and max / min of phi_rot60 -
    phi on the disk of radius c - 1 about the centre (c, c)."""
    r = np.arange(0, c, dtype=float)
    pa = bilinear(phi, c + 0 * r, c + r)
    pb = bilinear(phi, c - math.sqrt(3) / 2 * r, c + 0.5 * r)
    n = phi.shape[0]
    yy, xx = np.mgrid[0:n, 0:n].astype(float)
    th = math.pi / 3
    X = c + (xx - c) * math.cos(th) - (yy - c) * math.sin(th)
    Y = c + (xx - c) * math.sin(th) + (yy - c) * math.cos(th)
    disk = np.hypot(xx - c, yy - c) <= c - 1
    rot = bilinear(phi, np.clip(Y, 0, n - 1), np.clip(X, 0, n - 1))
    d = (rot - phi)[disk]
    return err_l2(pa, pb), float(d.max()), float(d.min())


def sec42(L, grad, precision=None, n=800, steps=100000, stream=None):
    """The sixfold run of Sec. 4.2; returns the paper's measures and the tip
    along +x."""
    precision = L.LBPF_FP64 if precision is None else precision
    prm = dict(SEC42)
    lam = prm.pop("lam")
    cr = [L.make_crystal(L.LBPF_AS_ANGLE, eps=0.05, q=6, phi0=0.0)]
    dom = L.make_domain(n, n, 1, lam=lam, crystals=cr, bc=L.LBPF_BC_WALL_X | L.LBPF_BC_WALL_Y, **prm)
    s = L.Solver(dom, L.LBPF_D2Q9_D2Q5, grad, precision, stream=stream)
    c = n // 2
    s.seed([(c, c, 0.0, 10.0, 0)])
    s.step(steps)
    phi = s.field(L.LBPF_FIELD_PHI)[0].astype(np.float64)
    tip = s.measure(c, c)[0]
    s.close()
    e, dmax, dmin = isotropy_measures(phi, c)
    return dict(grad="DD" if grad == L.LBPF_GRAD_DD else "FD", err_l2=e, rot60_max=dmax, rot60_min=dmin,
                tip_x=float(tip[0]), steps=steps, n=n)


def _crossing(vals):
    """Outermost phi = 0 crossing (linear interpolation) of samples at unit
    spacing; -1 when there is none."""
    best = -1.0
    for k in range(len(vals) - 1):
        if vals[k] >= 0 > vals[k + 1]:
            best = k + vals[k] / (vals[k] - vals[k + 1])
    return best


def slice_pairs(phi, which, c):
    """The two slices of Sec. 5.2 for dendrite `which` as matching point sets
    (phi[z, y, x]); returns (slice 1, slice 2 mapped by the symmetry)."""
    n = phi.shape[0]
    a = np.arange(-c, n - c)
    if which == "A":  # x = c (YZ) against y = c (XZ) rotated 90 degrees about z
        A_, B_ = np.meshgrid(a, a, indexing="ij")
        return phi[c + B_, c + A_, c], phi[c + B_, c, c + A_]
    if which == "C":  # normals (1, 1, 0) and (1, -1, 0), +-45 degrees about z
        A_, B_ = np.meshgrid(a, a, indexing="ij")
        return phi[c + B_, c - A_, c + A_], phi[c + B_, c + A_, c + A_]
    # B: normals (1, 1, 1) and (1, 1, -1), related by z -> -z about the centre
    A_, B_ = np.meshgrid(a, a, indexing="ij")
    D_ = -(A_ + B_)
    ok = np.abs(D_) <= c
    A_, B_, D_ = A_[ok], B_[ok], D_[ok]
    return phi[c + D_, c + B_, c + A_], phi[c - D_, c + B_, c + A_]


def sec52(L, which, precision=None, n=351, steps=None, stream=None):
    """A dendrite of Sec. 5.2 with its slice comparison and its tips along
    <100>, <110> and <111> from the centre."""
    precision = L.LBPF_FP32 if precision is None else precision
    form, default_steps = DENDRITES[which]
    steps = default_steps if steps is None else steps
    prm = dict(SEC52)
    lam = prm.pop("lam")
    dom = L.make_domain(n, n, n, lam=lam, crystals=[L.make_crystal(**form)], bc=7, **prm)
    s = L.Solver(dom, L.LBPF_D3Q15_D3Q7, L.LBPF_GRAD_DD, precision, stream=stream)
    c = n // 2
    s.seed([(c, c, c, 8.0, 0)])
    s.step(steps)
    phi = s.field(L.LBPF_FIELD_PHI).astype(np.float64)
    s.close()
    p1, p2 = slice_pairs(phi, which, c)
    k = np.arange(0, n - c)
    tips = {"100": _crossing(phi[c, c, c + k]), "110": _crossing(phi[c, c + k, c + k]) * math.sqrt(2),
            "111": _crossing(phi[c + k, c + k, c + k]) * math.sqrt(3)}
    return dict(dendrite=which, steps=steps, n=n, slice_max_diff=float(np.abs(p1 - p2).max()),
                slice_err_l2=err_l2(p1, p2), tips_lu=tips,
                solid_fraction=float(((1 + phi) / 2).mean()))
