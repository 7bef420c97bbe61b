"""Simulation-level isotropy contrast of Sec. 4.2 (Figs. 4-6), scaled down.

The paper grows a sixfold crystal (Eq. As_Theta, q = 6) and compares phi with
its 60-degree rotation, and the phi profiles along n_a = (1, 0) and
n_b = (1/2, -sqrt(3)/2) with the relative l2 error of Eq. (Error_L2): both are
much smaller with directional derivatives than with central differences
(x14 and x56 on the paper's 800^2 run; those ratios are context, not bars).
Here: the validated 2D parameter set of Sec. 3.4 (dx/W0 = 0.4, dt/tau0 =
0.008, kappa = 4, lambda*), Delta = 0.55 as in the LB+DD q = 6 run of
Sec. 4.2, on a 160^2 periodic box for 3000 steps, before the arms reach the
box edges.
"""
import numpy as np
import pytest


def run(O, grad, n=160, steps=3000):
    from scipy.ndimage import map_coordinates
    cr = O.make_crystal(O.AS_ANGLE, eps=0.05, q=6, phi0=0.0)
    p = O.make_params(O.D2Q9_D2Q5, n, n, 1, grad=grad, dx=0.4, dt=0.008, W0=1.0, tau0=1.0,
                      kappa=4.0, delta=0.55, crystals=[cr])
    o = O.Oracle(p).seed([[n // 2, n // 2, 0, 10.0, 0]])
    o.step(steps)
    phi = o.fields()[0][0]
    c = n // 2
    yy, xx = np.mgrid[0:n, 0:n].astype(float)
    th = np.pi / 3
    X = c + (xx - c) * np.cos(th) - (yy - c) * np.sin(th)
    Y = c + (xx - c) * np.sin(th) + (yy - c) * np.cos(th)
    rot = map_coordinates(phi, [Y, X], order=1, mode="wrap")
    mask = np.hypot(xx - c, yy - c) < 0.45 * n
    maxdiff = np.abs(rot - phi)[mask].max()
    r = np.arange(0, int(0.45 * n))
    pa = map_coordinates(phi, [c + 0 * r, c + r], order=1)
    pb = map_coordinates(phi, [c - np.sqrt(3) / 2 * r, c + 0.5 * r], order=1)
    err = np.sqrt(((pa - pb) ** 2).sum() / (pa ** 2).sum())
    return maxdiff, err, o.measure(c, c)[0][0]


def test_dd_beats_fd_on_sixfold_growth(orc):
    pytest.importorskip("scipy")
    O = orc
    dd = run(O, O.GRAD_DD)
    fd = run(O, O.GRAD_FD)
    assert dd[2] > 40 and fd[2] > 40  # the arms grew well past the seed radius
    assert dd[0] < 0.5 * fd[0], (dd, fd)
    assert dd[1] < 0.5 * fd[1], (dd, fd)
