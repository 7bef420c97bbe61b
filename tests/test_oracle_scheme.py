"""Pins of the oracle's time step (Secs. 3.1-3.2) against what the mathematics fixes.

* Uniform states reduce both schemes to the explicit Euler method for the ODE
  pair d(phi)/dt = Q_phi / tau0, du/dt = (1/2) d(phi)/dt (Eq. PhaseField_KarmaRappel
  and Eq. Temp_Ramirez without gradients).
* With phi uniform the heat scheme is linear: a Fourier mode evolves by an
  exact Q x Q propagator (grid-free, matrix power), and its decay rate tends
  to kappa k^2 (Eq. ThermalDiffusivity, Chapman-Enskog) as k dx -> 0.
* Small perturbations of phi = 0 along an axis with the <100> function give
  a_s = 1 + eps, N = 0 everywhere: the phase-field scheme, non-local term
  included, is then linear with an exact propagator, and its growth rate
  tends to (1 - W0^2 a_s^2 k^2) / (tau0 a_s^2), the linearisation of
  Eq. (PhaseField_KarmaRappel) with tau = tau0 a_s^2.
* A planar interface at u = 0 relaxes to the stationary profile
  tanh(x / (sqrt(2) W0 a_s)) of Eq. (PhaseField_KarmaRappel).
* sum(u - phi/2) is conserved on a periodic box (integral of Eq. Temp_Ramirez).
* A centred seed keeps the symmetry of the lattice point group.
* A z-uniform 3D run equals a 2D run on the projected lattices.
"""
from itertools import permutations, product

import numpy as np
import pytest

C1 = dict(dx=0.4, dt=0.008, W0=1.0, tau0=1.0, kappa=2.0, delta=0.3)
C2 = dict(dx=0.01, dt=1.5e-5, W0=0.0125, tau0=1.5625e-4, kappa=1.0, lam=10.0, delta=0.3)


def grid(nz, ny, nx):
    return np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")


@pytest.mark.parametrize("lat", [0, 1, 2, 3, 4])
def test_uniform_state_is_explicit_euler(orc, lat):
    O = orc
    D = O.lattice(lat, 0)[0]
    nz = 3 if D == 3 else 1
    p = O.make_params(lat, 4, 5, nz, dx=0.5, dt=0.01, W0=1.0, tau0=1.3, kappa=1.7, lam=2.5)
    o = O.Oracle(p)
    ph, uu = 0.3, -0.2
    shape = (nz, 5, 4)
    o.set_fields(np.full(shape, ph), np.full(shape, uu))
    q = 0.01 / 1.3
    for _ in range(30):
        o.step(1)
        Qphi = (ph - 2.5 * uu * (1 - ph * ph)) * (1 - ph * ph)
        ph_new = ph + q * Qphi
        uu = uu + 0.5 * (ph_new - ph)
        ph = ph_new
        phi, u, _ = o.fields()
        assert np.abs(phi - ph).max() < 1e-14 and np.abs(u - uu).max() < 1e-14


def heat_mode_run(O, lat, m, nsteps, kappa=0.9, dx=0.5, dt=0.05):
    D, e, w, e2 = O.lattice(lat, 1)
    n = (32, 24, 16 if D == 3 else 1)
    p = O.make_params(lat, *n, dx=dx, dt=dt, kappa=kappa, lam=1.0)
    z, y, x = grid(n[2], n[1], n[0])
    k = 2 * np.pi * np.array(m) / (np.array(n) * dx)
    th = (k[0] * x + k[1] * y + k[2] * z) * dx + 0.3
    o = O.Oracle(p).set_fields(-np.ones(x.shape), np.cos(th))
    return o, e, w, e2, k, th


@pytest.mark.parametrize("lat", [0, 1, 4])
def test_heat_scheme_exact_fourier_propagator(orc, lat):
    O = orc
    kappa, dx, dt = 0.9, 0.5, 0.05
    m = (2, 1, 1)
    o, e, w, e2, k, th = heat_mode_run(O, lat, m, 0, kappa, dx, dt)
    eta = kappa * dt / (e2 * dx * dx) + 0.5
    om = 1 - 1 / eta
    ph = np.exp(-1j * dx * (e @ k))
    M = ph[:, None] * (om * np.eye(len(w)) + (1 - om) * np.outer(w, np.ones(len(w))))
    v = w.astype(complex)
    for step in range(1, 41):
        o.step(1)
        v = M @ v
        if step % 10 == 0:
            want = np.real(v.sum() * np.exp(1j * th))
            _, u, _ = o.fields()
            assert np.abs(u - want).max() < 1e-13, step
            phi = o.fields()[0]
            assert np.abs(phi + 1.0).max() < 1e-14


@pytest.mark.parametrize("lat", [0, 1])
def test_heat_scheme_diffusivity(orc, lat):
    """Long-wave decay rate equals kappa |k|^2 (the kappa-eta relation)."""
    O = orc
    kappa, dx, dt = 0.9, 0.5, 0.05
    o, e, w, e2, k, th = heat_mode_run(O, lat, (1, 0, 0), 0, kappa, dx, dt)
    amps = []
    for _ in range(3):
        o.step(50)
        u = o.fields()[1]
        amps.append((u * np.cos(th)).sum() / (np.cos(th) ** 2).sum())
    rate = -np.log(amps[2] / amps[1]) / (50 * dt)
    assert abs(rate / (kappa * (k @ k)) - 1) < 0.01, rate / (kappa * (k @ k))


def phase_mode_setup(O, lat, eps, kx_mult, dx=0.4, dt=0.008, W0=1.0, tau0=1.0):
    D = O.lattice(lat, 0)[0]
    n = (40, 3, 3 if D == 3 else 1)
    p = O.make_params(lat, *n, dx=dx, dt=dt, W0=W0, tau0=tau0, kappa=1.0, lam=0.0,
                      crystals=[O.make_crystal(O.AS_CUBIC100, eps=eps)])
    z, y, x = grid(n[2], n[1], n[0])
    k = 2 * np.pi * kx_mult / (n[0] * dx)
    th = k * x * dx + 0.37  # no grid point with zero gradient
    amp = 1e-7
    o = O.Oracle(p).set_fields(amp * np.cos(th), np.zeros(x.shape))
    return o, p, k, th, amp


@pytest.mark.parametrize("lat", [0, 1, 3])
@pytest.mark.parametrize("eps", [0.0, 0.08])
def test_phase_scheme_exact_linear_propagator(orc, lat, eps):
    O = orc
    dx, dt, W0, tau0 = 0.4, 0.008, 1.0, 1.0
    o, p, k, th, amp = phase_mode_setup(O, lat, eps, 3, dx, dt, W0, tau0)
    D, e, w, e2 = O.lattice(lat, 0)
    a = 1 + eps
    Dphi = W0 * W0 / tau0 * dt / (dx * dx)
    eta = a * a * Dphi / e2 + 0.5
    q = dt / tau0
    Q = len(w)
    sh = np.exp(1j * k * dx * e[:, 0])
    M = (np.diag(1 / sh) @ ((1 - 1 / eta) * np.eye(Q) - (1 - a * a) * np.diag(sh)
                            + (1 / eta + q) * np.outer(w, np.ones(Q)))) / (a * a)
    v = w.astype(complex) * amp
    for step in range(1, 61):
        o.step(1)
        v = M @ v
        if step % 20 == 0:
            want = np.real(v.sum() * np.exp(1j * th))
            phi = o.fields()[0]
            assert np.abs(phi - want).max() < 1e-12 * np.abs(want).max(), step


@pytest.mark.parametrize("eps", [0.0, 0.1])
def test_phase_scheme_growth_rate(orc, eps):
    """Long-wave modes of phi = 0 grow at sigma(k) = (1 - W0^2 a^2 k^2)/(tau0 a^2),
    the linearisation of Eq. (PhaseField_KarmaRappel) with tau = tau0 a_s^2:
    sigma(k -> 0) pins the kinetic factor 1/a_s^2, and sigma(k1) - sigma(k2)
    = W0^2 (k2^2 - k1^2) / tau0 pins the diffusivity W0^2/tau0 of Eq.
    (LBE_RelaxationTime), independently of a_s."""
    O = orc
    dx, dt, nx = 0.4, 0.008, 200
    a = 1 + eps
    sig = {}
    for m in (1, 4):
        p = O.make_params(O.D2Q9_D2Q5, nx, 3, 1, dx=dx, dt=dt, W0=1.0, tau0=1.0, kappa=1.0, lam=0.0,
                          crystals=[O.make_crystal(O.AS_CUBIC100, eps=eps)])
        z, y, x = grid(1, 3, nx)
        k = 2 * np.pi * m / (nx * dx)
        th = k * x * dx + 0.37
        o = O.Oracle(p).set_fields(1e-7 * np.cos(th), np.zeros(x.shape))
        A = []
        for _ in range(3):
            o.step(100)
            phi = o.fields()[0]
            A.append((phi * np.cos(th)).sum() / (np.cos(th) ** 2).sum())
        sig[m] = ((A[2] / A[1]) ** (1 / 100) - 1) / dt  # explicit Euler per-step rate
        sig[m, "k"] = k
    k1, k6 = sig[1, "k"], sig[4, "k"]
    assert abs(sig[1] / (1 / a ** 2 - k1 ** 2) - 1) < 0.005, sig[1]
    assert abs((sig[1] - sig[4]) / (k6 ** 2 - k1 ** 2) - 1) < 0.03, (sig[1] - sig[4], k6 ** 2 - k1 ** 2)


@pytest.mark.parametrize("eps", [0.0, 0.1])
def test_planar_interface_width(orc, eps):
    O = orc
    dx, W0 = 0.25, 1.0
    nx = 160
    p = O.make_params(O.D2Q9_D2Q5, nx, 4, 1, dx=dx, dt=0.01, W0=W0, tau0=1.0, kappa=1.0, lam=0.0,
                      crystals=[O.make_crystal(O.AS_CUBIC100, eps=eps)])
    z, y, x = grid(1, 4, nx)
    c, R = nx / 2, 40.0
    phi0 = np.tanh((R - np.abs(x - c + 0.5)) * dx / (np.sqrt(2) * W0))
    o = O.Oracle(p).set_fields(phi0, np.zeros(x.shape))
    o.step(4000)  # 40 tau0
    phi = o.fields()[0][0, 1]
    i0 = np.where((phi[:-1] >= 0) & (phi[1:] < 0))[0][-1]
    xc = i0 + phi[i0] / (phi[i0] - phi[i0 + 1])
    # for tanh(x / (sqrt2 W)), the integral of 1 - phi^2 across one interface is 2 sqrt2 W
    W = (1 - phi ** 2).sum() * dx / (2 * 2 * np.sqrt(2))
    assert abs(W / (W0 * (1 + eps)) - 1) < 0.005, W
    assert abs(xc - (c + R - 0.5)) < 0.05
    # whole profile against the stationary tanh
    xs = np.arange(nx)
    want = np.tanh((R - np.abs(xs - c + 0.5)) * dx / (np.sqrt(2) * W0 * (1 + eps)))
    assert np.abs(phi - want).max() < 5e-3


def c1_oracle(O, n=64, grad=0, steps=0, kind=None, **kw):
    cr = kind if kind is not None else O.make_crystal(O.AS_CUBIC100, eps=0.05)
    p = O.make_params(O.D2Q9_D2Q5, n, n, 1, grad=grad, crystals=[cr], **C1)
    o = O.Oracle(p).seed([[n // 2, n // 2, 0, 10.0, 0]])
    if steps:
        o.step(steps)
    return o


def test_seed_profile(orc):
    O = orc
    o = c1_oracle(O)
    phi, u, I = o.fields()
    assert phi[0, 32, 42] == 0.0  # d = R
    assert abs(phi[0, 32, 32] - np.tanh(10 * 0.4 / np.sqrt(2))) < 1e-15
    assert np.all(u == -0.3) and np.all(I == 1)


def test_conservation_c1(orc):
    O = orc
    o = c1_oracle(O, 64)
    _, _, c0 = o.measure(32, 32)
    o.step(1000)
    tip, sf, c1 = o.measure(32, 32)
    assert abs(c1 - c0) <= 1e-12 * abs(c0)
    assert tip[0] > 11  # the undercooled seed grows


def sym_ops_2d():
    for t, sx, sy in product((False, True), (1, -1), (1, -1)):
        yield t, sx, sy


def apply_2d(a, t, sx, sy):
    n = a.shape[-1]
    idx = lambda s: (s * np.arange(n)) % n
    b = a[..., idx(sy), :][..., :, idx(sx)]
    return np.swapaxes(b, -1, -2) if t else b


@pytest.mark.parametrize("grad", [0, 1])
def test_symmetry_2d(orc, grad):
    O = orc
    o = c1_oracle(O, 64, grad=grad, steps=400)
    phi, u, _ = o.fields()
    # centre 32: reflect about it by shifting the centre to the origin
    phc, uc = np.roll(phi, (-32, -32), (-2, -1)), np.roll(u, (-32, -32), (-2, -1))
    for op in sym_ops_2d():
        assert np.abs(apply_2d(phc, *op) - phc).max() < 1e-12
        assert np.abs(apply_2d(uc, *op) - uc).max() < 1e-12
    assert np.abs(phi - np.roll(phi, 1, -1)).max() > 0.1  # not trivially uniform


@pytest.mark.parametrize("lat", [1, 2, 3])
def test_symmetry_3d(orc, lat):
    O = orc
    n = 20
    p = O.make_params(lat, n, n, n, crystals=[O.make_crystal(O.AS_CUBIC100, eps=0.05)], **C2)
    o = O.Oracle(p).seed([[10, 10, 10, 5.0, 0]])
    o.step(60)
    phi, u, _ = o.fields()
    phc = np.roll(phi, (-10, -10, -10), (0, 1, 2))
    uc = np.roll(u, (-10, -10, -10), (0, 1, 2))
    idx = lambda s: (s * np.arange(n)) % n
    for perm in permutations(range(3)):
        for s in product((1, -1), repeat=3):
            for f in (phc, uc):
                g = np.transpose(f, perm)
                g = g[idx(s[0])][:, idx(s[1])][:, :, idx(s[2])]
                assert np.abs(g - f).max() < 1e-12


@pytest.mark.parametrize("lat3", [1, 2, 3])
@pytest.mark.parametrize("kind", ["cubic", "y66"])
def test_z_uniform_3d_equals_2d(orc, lat3, kind):
    O = orc
    cr = O.make_crystal(O.AS_CUBIC100, eps=0.05) if kind == "cubic" else O.make_crystal(O.AS_Y66, eps=0.05)
    n = 32
    kw = dict(dx=0.01, dt=1.5e-5, W0=0.0125, tau0=1.5625e-4, kappa=0.7, lam=10.0)
    p2 = O.make_params(O.D2Q9_D2Q5P, n, n, 1, crystals=[cr], **kw)
    p3 = O.make_params(lat3, n, n, 3, crystals=[cr], **kw)
    z, y, x = grid(1, n, n)
    r = np.sqrt((x - 15.6) ** 2 + (y - 16.2) ** 2)
    phi0 = np.tanh((6 - r) * 0.01 / (np.sqrt(2) * 0.0125))
    u0 = np.full(phi0.shape, -0.3)
    o2 = O.Oracle(p2).set_fields(phi0, u0)
    o3 = O.Oracle(p3).set_fields(np.repeat(phi0, 3, 0), np.repeat(u0, 3, 0))
    o2.step(150)
    o3.step(150)
    f2, f3 = o2.fields(), o3.fields()
    for a, b in zip(f2[:2], f3[:2]):
        assert np.abs(b - a).max() < 1e-12
    assert np.abs(f2[0] - phi0).max() > 1e-2  # the run did something
