"""Python access to the FP64 CPU oracle (``lbpf_oracle.c``).

Test infrastructure only: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the product library never does.  It
shares no code with the CUDA path.

The oracle follows Younsi & Cartalade (arXiv:1606.09432): the heat scheme of
Sec. 3.1, the phase-field scheme of Sec. 3.2, the lattices of Sec. 3.3
(Table 1), the gradient operators of Sec. 4.2 and the anisotropy functions of
Secs. 2 and 4.1, in physical units and double precision.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbpf_oracle.c")
_LIB = os.path.join(_HERE, f"liborc.{platform.machine()}.so")

MAXC = 16

# Lattice pairs, in the oracle's numbering.
D2Q9_D2Q5, D3Q15_D3Q7, D3Q19_D3Q7, D3Q27_D3Q7, D2Q9_D2Q5P = range(5)
# Anisotropy kinds.
AS_CUBIC100, AS_ANGLE, AS_Y66, AS_HOYT110, AS_S111 = range(5)
# Gradient operators.
GRAD_DD, GRAD_FD = 0, 1
# Boundary bits: zero-flux walls at both ends of an axis (0: periodic box).
WALL_X, WALL_Y, WALL_Z = 1, 2, 4

# Thin-interface coefficients, Eqs. (Capillary-Length) and (Kinetic-Coeff):
# a1 = 5 sqrt(2) / 8 and a2 ~ 0.6267 (the paper's lambda* = 1.59566 kappa
# at W0 = tau0 = 1 is 1 / 0.6267).
A1 = 5.0 * math.sqrt(2.0) / 8.0
A2 = 0.6267


def lambda_star(kappa: float, tau0: float, W0: float) -> float:
    """Coupling constant that cancels the kinetic coefficient (beta = 0):
    lambda* = kappa tau0 / (a2 W0^2), Eq. (Kinetic-Coeff) set to zero."""
    return kappa * tau0 / (A2 * W0 * W0)


def capillary_length(W0: float, lam: float) -> float:
    """d0 = a1 W0 / lambda, Eq. (Capillary-Length)."""
    return A1 * W0 / lam


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library beside its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class Crystal(C.Structure):
    _fields_ = [("kind", C.c_int), ("eps", C.c_double), ("gamma", C.c_double),
                ("q", C.c_int), ("phi0", C.c_double)]


class Params(C.Structure):
    _fields_ = [("lattice", C.c_int), ("grad", C.c_int),
                ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("bc", C.c_int),
                ("dx", C.c_double), ("dt", C.c_double), ("W0", C.c_double),
                ("tau0", C.c_double), ("kappa", C.c_double), ("lam", C.c_double),
                ("delta", C.c_double), ("xi", C.c_double),
                ("n_crystals", C.c_int), ("crystals", Crystal * MAXC), ("adv", C.c_double * 3)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d = C.POINTER(C.c_double)
        i = C.POINTER(C.c_int)
        _lib.orc_create.restype = C.c_void_p
        _lib.orc_create.argtypes = [C.POINTER(Params)]
        _lib.orc_destroy.argtypes = [C.c_void_p]
        _lib.orc_seed.argtypes = [C.c_void_p, d, C.c_int]
        _lib.orc_set_fields.argtypes = [C.c_void_p, d, d, i]
        _lib.orc_set_populations.argtypes = [C.c_void_p, d, d]
        _lib.orc_step.argtypes = [C.c_void_p, C.c_int]
        _lib.orc_steps_done.restype = C.c_long
        _lib.orc_steps_done.argtypes = [C.c_void_p]
        _lib.orc_get_fields.argtypes = [C.c_void_p, d, d, i]
        _lib.orc_get_populations.argtypes = [C.c_void_p, d, d]
        _lib.orc_get_anisotropy.argtypes = [C.c_void_p, d]
        _lib.orc_anisotropy_field.argtypes = [C.c_void_p, d]
        _lib.orc_measure.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, d, d, d]
        _lib.orc_lattice.argtypes = [C.c_int, C.c_int, i, i, i, d, d]
        _lib.orc_gradient.argtypes = [C.POINTER(Params), d, d]
        _lib.orc_anisotropy.argtypes = [C.POINTER(Crystal), C.c_int, C.c_double, d, d, d]
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def lattice(lat: int, which: int):
    """(D, e[Q,3], w[Q], e2) of the phase-field (which=0) or temperature
    (which=1) lattice of a lattice pair."""
    D, Q = C.c_int(), C.c_int()
    e = np.zeros(27 * 3, dtype=np.int32)
    w = np.zeros(27)
    e2 = C.c_double()
    if lib().orc_lattice(lat, which, C.byref(D), C.byref(Q), _ip(e), _dp(w), C.byref(e2)):
        raise ValueError("unknown lattice")
    q = Q.value
    return D.value, e[: 3 * q].reshape(q, 3).copy(), w[:q].copy(), e2.value


def make_crystal(kind=AS_CUBIC100, eps=0.0, gamma=0.0, q=4, phi0=0.0) -> Crystal:
    return Crystal(kind, eps, gamma, q, phi0)


def make_params(lattice_pair, nx, ny, nz=1, *, grad=GRAD_DD, dx=1.0, dt=1.0, W0=1.0, tau0=1.0,
                kappa=1.0, lam=None, delta=0.0, xi=1e-7, crystals=(None,), bc=0, adv=(0.0, 0.0, 0.0)) -> Params:
    p = Params()
    p.lattice = lattice_pair
    p.grad = grad
    p.nx, p.ny, p.nz = nx, ny, nz
    p.bc = bc
    for a in range(3):
        p.adv[a] = float(adv[a])
    p.dx, p.dt, p.W0, p.tau0, p.kappa = dx, dt, W0, tau0, kappa
    p.lam = lambda_star(kappa, tau0, W0) if lam is None else lam
    p.delta = delta
    p.xi = xi
    cl = [c if c is not None else make_crystal() for c in crystals]
    if not 1 <= len(cl) <= MAXC:
        raise ValueError("1..16 crystals")
    p.n_crystals = len(cl)
    for k, c in enumerate(cl):
        p.crystals[k] = c
    return p


def gradient(p: Params, phi: np.ndarray) -> np.ndarray:
    """Physical gradient of a (nz, ny, nx) field by the operator p.grad."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    G = np.zeros(phi.shape + (3,))
    lib().orc_gradient(C.byref(p), _dp(phi), _dp(G))
    return G


def anisotropy(crystal: Crystal, D: int, G, dx: float = 1.0):
    """(a_s, N) for a physical gradient G (3-vector)."""
    Gv = np.ascontiguousarray(np.asarray(G, dtype=np.float64).reshape(3))
    N = np.zeros(3)
    a = C.c_double()
    if lib().orc_anisotropy(C.byref(crystal), D, dx, _dp(Gv), C.byref(a), _dp(N)):
        raise ValueError("invalid anisotropy kind for this dimension")
    return a.value, N


class Oracle:
    """One periodic domain advanced by the FP64 reference scheme."""

    def __init__(self, p: Params):
        self.p = p
        self.shape = (p.nz, p.ny, p.nx)
        self.n = p.nx * p.ny * p.nz
        self.Qg = lattice(p.lattice, 0)[1].shape[0]
        self.Qu = lattice(p.lattice, 1)[1].shape[0]
        self._h = lib().orc_create(C.byref(p))
        if not self._h:
            raise ValueError("invalid oracle parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def seed(self, seeds):
        """seeds: rows (x, y, z, R, crystal) in lattice units."""
        s = np.ascontiguousarray(np.asarray(seeds, dtype=np.float64).reshape(-1, 5))
        if lib().orc_seed(self._h, _dp(s), s.shape[0]):
            raise ValueError("bad seeds")
        return self

    def set_fields(self, phi, u, I=None):
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(self.shape)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(self.shape)
        Ip = None
        if I is not None:
            Iarr = np.ascontiguousarray(I, dtype=np.int32).reshape(self.shape)
            Ip = _ip(Iarr)
        lib().orc_set_fields(self._h, _dp(phi), _dp(u), Ip)
        return self

    def set_populations(self, g, f):
        g = np.ascontiguousarray(g, dtype=np.float64).reshape((self.Qg,) + self.shape)
        f = np.ascontiguousarray(f, dtype=np.float64).reshape((self.Qu,) + self.shape)
        lib().orc_set_populations(self._h, _dp(g), _dp(f))
        return self

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))
        return self

    @property
    def steps_done(self) -> int:
        return lib().orc_steps_done(self._h)

    def fields(self):
        phi = np.zeros(self.shape)
        u = np.zeros(self.shape)
        I = np.zeros(self.shape, dtype=np.int32)
        lib().orc_get_fields(self._h, _dp(phi), _dp(u), _ip(I))
        return phi, u, I

    def populations(self):
        g = np.zeros((self.Qg,) + self.shape)
        f = np.zeros((self.Qu,) + self.shape)
        lib().orc_get_populations(self._h, _dp(g), _dp(f))
        return g, f

    def anisotropy_field(self):
        """a_s used by the last step (from the phase field before it)."""
        a = np.zeros(self.shape)
        lib().orc_get_anisotropy(self._h, _dp(a))
        return a

    def current_anisotropy(self):
        """a_s of the current phase field and index field."""
        a = np.zeros(self.shape)
        lib().orc_anisotropy_field(self._h, _dp(a))
        return a

    def measure(self, cx: int, cy: int, cz: int = 0):
        tip = np.zeros(6)
        sf = C.c_double()
        cs = C.c_double()
        lib().orc_measure(self._h, cx, cy, cz, _dp(tip), C.byref(sf), C.byref(cs))
        return tip, sf.value, cs.value


# ---------------------------------------------------------------------------
# Tip kinetics.  The paper defines the tip velocity V_p and its dimensionless
# form V_p d0 / kappa (Sec. 3.4) but neither the tip position nor the tip
# radius.  Readings: the tip position is the outermost phi = 0 crossing on the
# axis ray (orc_measure); the tip velocity is the least-squares slope of the
# tip position over time; the tip radius is rho = -1/(2b) from the
# least-squares fit x_c(j) = a + b j^2 of the crossings on the rays parallel to
# the axis at transverse offsets |j| <= J (in 3D, the mean of the two
# transverse planes).
# ---------------------------------------------------------------------------

def tip_velocity(times, positions):
    """Least-squares slope of positions over times (a library fit as one step)."""
    t = np.asarray(times, dtype=np.float64)
    x = np.asarray(positions, dtype=np.float64)
    return float(np.polyfit(t, x, 1)[0])


def _reflect(v, n):
    while v < 0 or v > n - 1:
        v = -v if v < 0 else 2 * (n - 1) - v
    return v


def ray_crossing(phi, centre, axis, sign, offsets, bc=0):
    """Outermost phi = 0 crossing (linear interpolation) along the ray from
    `centre` shifted by `offsets` (dict axis -> shift), in direction sign along
    `axis`, over half the box (up to the wall along a walled axis, bc bit
    1 << axis; offsets beyond a wall are reflected); -1 when there is none.
    phi is (nz, ny, nx)."""
    shape = phi.shape[::-1]  # (nx, ny, nz)
    c = list(centre)
    for ax, sh in offsets.items():
        c[ax] = _reflect(c[ax] + sh, shape[ax]) if bc >> ax & 1 else (c[ax] + sh) % shape[ax]
    length = (shape[axis] - 1 - c[axis] if sign > 0 else c[axis]) if bc >> axis & 1 else shape[axis] // 2
    best = -1.0
    for k in range(length):
        p0i, p1i = list(c), list(c)
        p0i[axis] = (c[axis] + sign * k) % shape[axis]
        p1i[axis] = (c[axis] + sign * (k + 1)) % shape[axis]
        p0 = phi[p0i[2], p0i[1], p0i[0]]
        p1 = phi[p1i[2], p1i[1], p1i[0]]
        if p0 >= 0.0 and p1 < 0.0:
            best = k + p0 / (p0 - p1)
    return best


def tip_radius(phi, centre, direction, J=3, bc=0):
    """Tip radius (lattice units) of the tip along direction 0..5
    (+x, -x, +y, -y, +z, -z) from the crossings at transverse offsets |j| <= J
    (bc: wall bits, see ray_crossing)."""
    axis, sign = direction // 2, (1 if direction % 2 == 0 else -1)
    dim = 3 if phi.shape[0] > 1 else 2
    planes = [a for a in range(dim) if a != axis]
    rhos = []
    for tr in planes:
        js, xs = [], []
        for j in range(-J, J + 1):
            x = ray_crossing(phi, centre, axis, sign, {tr: j}, bc)
            if x >= 0:
                js.append(j * j)
                xs.append(x)
        if len(js) >= 3:
            b = np.polyfit(np.array(js, float), np.array(xs), 1)[0]
            rhos.append(-1.0 / (2.0 * b))
    return float(np.mean(rhos)) if rhos else -1.0
