"""Pins of the tip-kinetics readings (parity unpinned by the paper: it
defines only the tip velocity V_p, Sec. 3.4).  Closed forms: a parabolic tip
phi = x_tip - x - y^2/(2 rho) has its crossings exactly on x_c(j) = x_tip -
j^2/(2 rho) (phi is linear along x, so linear interpolation is exact), giving
rho back exactly; a paraboloid in 3D likewise; a tip moving at constant speed
gives its speed; a circle of radius R gives rho ~ R."""
import numpy as np
import pytest


def test_parabolic_tip_2d(orc):
    O = orc
    n = 96
    y, x = np.mgrid[0:n, 0:n].astype(float)
    c = 40
    for rho, xt in ((7.5, 20.3), (15.0, 11.7)):
        phi = (xt - (x - c)) - (y - c) ** 2 / (2 * rho)
        phi = phi[None]
        assert abs(O.tip_radius(phi, (c, c, 0), 0, J=3) - rho) < 1e-9
        assert abs(O.ray_crossing(phi, (c, c, 0), 0, 1, {}) - xt) < 1e-12


def test_paraboloid_tip_3d(orc):
    O = orc
    n = 48
    z, y, x = np.mgrid[0:n, 0:n, 0:n].astype(float)
    c = 20
    rho = 6.0
    phi = (9.4 - (z - c)) - ((x - c) ** 2 + (y - c) ** 2) / (2 * rho)
    assert abs(O.tip_radius(phi, (c, c, c), 4, J=3) - rho) < 1e-9
    # -x tip of a paraboloid opening along +x
    phi2 = (7.2 + (x - c)) - ((y - c) ** 2 + (z - c) ** 2) / (2 * 4.0)
    assert abs(O.tip_radius(phi2, (c, c, c), 1, J=2) - 4.0) < 1e-9


def test_circle_radius(orc):
    O = orc
    n = 128
    y, x = np.mgrid[0:n, 0:n].astype(float)
    R = 30.0
    phi = np.tanh((R - np.hypot(x - 64, y - 64)) / 2.0)[None]
    # approximate: linear interpolation of a curved tanh profile biases the
    # crossings by ~1e-2 sites, a few percent of the small j^2 term
    assert abs(O.tip_radius(phi, (64, 64, 0), 2, J=3) / R - 1) < 0.06


def test_tip_velocity_constant_speed(orc):
    O = orc
    t = np.arange(10) * 0.4
    assert abs(O.tip_velocity(t, 3.0 + 0.125 * t) - 0.125) < 1e-14
