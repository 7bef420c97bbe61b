"""Pins of the oracle's advection-diffusion form of the heat scheme (Sec.
3.1): the equilibrium f_i^(0) = w_i u [1 + e^{-2} e_i . v dt/dx] turns the
scheme into one for du/dt = kappa lap u - div(u v).

* The moments of that equilibrium are those Sec. 3.1 states: u,
  v u dt/dx and e^2 u I.
* With phi uniform the scheme is linear: a Fourier mode of u evolves by an
  exact Q x Q propagator whose collision matrix carries the advective term.
* Its long-wave behaviour is the continuum equation's: the mode travels with
  phase speed v . k / |k| and decays at the rate kappa |k|^2.
"""
import numpy as np
import pytest


def grid(nz, ny, nx):
    return np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")


@pytest.mark.parametrize("lat", [0, 1, 2])
def test_advective_equilibrium_moments(orc, lat):
    O = orc
    D, e, w, e2 = O.lattice(lat, 1)
    nz = 4 if D == 3 else 1
    dx, dt = 0.5, 0.05
    v = (0.8, -0.5, 0.3 if D == 3 else 0.0)
    p = O.make_params(lat, 5, 6, nz, dx=dx, dt=dt, kappa=0.9, lam=1.0, adv=v)
    rng = np.random.default_rng(2)
    u = rng.standard_normal((nz, 6, 5))
    f = O.Oracle(p).set_fields(-np.ones(u.shape), u).populations()[1]
    e = e.astype(float)
    assert np.abs(f.sum(axis=0) - u).max() <= 1e-14
    m1 = np.einsum("qa,qzyx->zyxa", e, f)
    assert np.abs(m1 - np.asarray(v)[:3] * (dt / dx) * u[..., None]).max() <= 1e-14
    m2 = np.einsum("qa,qb,qzyx->zyxab", e, e, f)
    want = e2 * u[..., None, None] * np.diag([1.0, 1.0, 1.0 if D == 3 else 0.0])
    assert np.abs(m2 - want).max() <= 1e-14


@pytest.mark.parametrize("lat", [0, 1])
def test_advection_exact_fourier_propagator(orc, lat):
    O = orc
    D, e, w, e2 = O.lattice(lat, 1)
    kappa, dx, dt = 0.9, 0.5, 0.05
    v = np.array([1.3, -0.7, 0.4 if D == 3 else 0.0])
    n = (32, 24, 16 if D == 3 else 1)
    p = O.make_params(lat, *n, dx=dx, dt=dt, kappa=kappa, lam=1.0, adv=v)
    z, y, x = grid(n[2], n[1], n[0])
    k = 2 * np.pi * np.array((2, 1, 1)) / (np.array(n) * dx)
    th = (k[0] * x + k[1] * y + k[2] * z) * dx + 0.3
    o = O.Oracle(p).set_fields(-np.ones(x.shape), np.cos(th))
    eta = kappa * dt / (e2 * dx * dx) + 0.5
    om = 1 - 1 / eta
    weq = w * (1 + (e @ v) * (dt / dx) / e2)  # equilibrium per unit u
    ph = np.exp(-1j * dx * (e @ k))
    M = ph[:, None] * (om * np.eye(len(w)) + (1 - om) * np.outer(weq, np.ones(len(w))))
    a = weq.astype(complex)  # the mode starts at equilibrium
    for step in range(1, 41):
        o.step(1)
        a = M @ a
        if step % 10 == 0:
            want = np.real(a.sum() * np.exp(1j * th))
            assert np.abs(o.fields()[1] - want).max() < 1e-13, step


@pytest.mark.parametrize("lat", [0, 1])
def test_advection_long_wave_limit(orc, lat):
    """A long wave along x travels at v_x and decays at kappa k^2 (the
    equilibrium is linear in v, so the decay carries an O(v^2 dt) numerical
    diffusion: 2.5 % at v = 2 here; v = 0.5 makes it negligible)."""
    O = orc
    kappa, dx, dt = 0.9, 0.5, 0.02
    vx = 0.5
    D = O.lattice(lat, 1)[0]
    n = (128, 3, 3 if D == 3 else 1)
    p = O.make_params(lat, *n, dx=dx, dt=dt, kappa=kappa, lam=1.0, adv=(vx, 0.0, 0.0))
    z, y, x = grid(n[2], n[1], n[0])
    k = 2 * np.pi / (n[0] * dx)
    th = k * x * dx
    o = O.Oracle(p).set_fields(-np.ones(x.shape), np.cos(th))
    steps = 400
    o.step(40)  # past the initial transient of the non-equilibrium moments
    u0 = o.fields()[1]
    o.step(steps)
    u1 = o.fields()[1]
    c0 = (u0 * np.exp(-1j * th)).sum()
    c1 = (u1 * np.exp(-1j * th)).sum()
    rate = c1 / c0
    t = steps * dt
    speed = -np.angle(rate) / (k * t)
    decay = -np.log(np.abs(rate)) / t
    assert abs(speed / vx - 1) < 2e-3, speed
    assert abs(decay / (kappa * k * k) - 1) < 5e-3, decay / (kappa * k * k)
