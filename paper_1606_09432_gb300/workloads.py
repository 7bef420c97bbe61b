"""Seeded synthetic workloads: domain sizes, model parameters and seed
layouts of the configurations this library is exercised on.

These are inputs only (numbers and seeded random draws); they contain none of
the solver's arithmetic.  Parameters are physical (dx, dt, W0, tau0, kappa);
lam = None asks each side for lambda* (beta = 0).
"""
from __future__ import annotations

import math

# 2D validated parameter set of the paper's Sec. 3.4 (dx/W0 = 0.4,
# dt/tau0 = 0.008, W0 = tau0 = 1), with kappa = 2.
C1_PARAMS = dict(dx=0.4, dt=0.008, W0=1.0, tau0=1.0, kappa=2.0, lam=None, delta=0.3)
# 3D parameter set of the paper's Sec. 5.2 (dx = 0.01, dt = 1.5e-5,
# W0 = 0.0125, tau0 = 1.5625e-4, lambda = 10, kappa = 1).
C3D_PARAMS = dict(dx=0.01, dt=1.5e-5, W0=0.0125, tau0=1.5625e-4, kappa=1.0, lam=10.0)


def c1(n=128):
    """2D plain method: n^2 periodic, D2Q9/D2Q5, <100> eps = 0.05, Delta = 0.3,
    one centred seed of radius 10 sites."""
    return dict(shape=(1, n, n), params=dict(C1_PARAMS), aniso=dict(kind=0, eps=0.05),
                seeds=[(n // 2, n // 2, 0, 10.0, 0)], centre=(n // 2, n // 2, 0))


def c2(n=256, delta=0.3):
    """3D single crystal: n^3 periodic, <100> eps = 0.05, centred seed of radius 8."""
    return dict(shape=(n, n, n), params=dict(C3D_PARAMS, delta=delta), aniso=dict(kind=0, eps=0.05),
                seeds=[(n // 2, n // 2, n // 2, 8.0, 0)], centre=(n // 2, n // 2, n // 2))


def c3(n=512, eps=0.0, gamma=-0.02):
    """3D precision form: n^3, <110>/<111> form of Eq. (As_MatSci), Delta = 0.4."""
    return dict(shape=(n, n, n), params=dict(C3D_PARAMS, delta=0.4), aniso=dict(kind=3, eps=eps, gamma=gamma),
                seeds=[(n // 2, n // 2, n // 2, 8.0, 0)], centre=(n // 2, n // 2, n // 2))


def octant(n=351, eps=0.0, gamma=-0.02, delta=0.25, radius=8.0):
    """The octant run of the paper's Sec. 5.3 (dendrite B): n^3 nodes with
    zero-flux walls on all six faces (bc = 7), the seed at the origin on three
    of them, the 3D parameter set of Sec. 5.2, the <110> form of Eq.
    (As_MatSci) with (eps, gamma) = (0, -0.02), Delta = 0.25.  The paper does
    not state the seed radius of its 3D runs; 8 sites as in the other 3D
    configurations."""
    return dict(shape=(n, n, n), params=dict(C3D_PARAMS, delta=delta), aniso=dict(kind=3, eps=eps, gamma=gamma),
                seeds=[(0.0, 0.0, 0.0, radius, 0)], centre=(0, 0, 0), bc=7)


class SplitMix64:
    """SplitMix64 generator (Steele, Lea, Flood 2014)."""

    def __init__(self, seed: int):
        self.s = seed & 0xFFFFFFFFFFFFFFFF

    def next(self) -> int:
        self.s = (self.s + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        return z ^ (z >> 31)

    def uniform(self, a=0.0, b=1.0) -> float:
        return a + (b - a) * ((self.next() >> 11) * (1.0 / 9007199254740992.0))

    def randint(self, a: int, b: int) -> int:
        """Uniform integer in [a, b]."""
        return a + int(self.uniform() * (b - a + 1))


# 2D multi-crystal batch parameters (dx/W0 = 5e-3/0.012, dt/tau0 = 5e-6/1e-4,
# lambda = 10, kappa = 0.7), the paper's Sec. 4.3 set.
C4_PARAMS = dict(dx=5e-3, dt=5e-6, W0=0.012, tau0=1e-4, kappa=0.7, lam=10.0)


def c4(n_domains=64, seed=1606094320, lmin=128, lmax=1024, max_seeds=12):
    """Batched 2D multi-crystal domains: side L ~ U{lmin..lmax}, 1..max_seeds
    seeds of radius U[4, 10] at non-overlapping random positions, per-crystal
    orientation theta ~ U[0, pi/2), eps ~ U[0.01, 0.07], Delta ~ U[0.2, 0.6]."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(n_domains):
        L = rng.randint(lmin, lmax)
        ns = rng.randint(1, max_seeds)
        delta = rng.uniform(0.2, 0.6)
        seeds, crystals = [], []
        tries = 0
        while len(seeds) < ns and tries < 10000:
            tries += 1
            r = rng.uniform(4.0, 10.0)
            x, y = rng.uniform(0, L), rng.uniform(0, L)
            ok = True
            for (sx, sy, _, sr, _) in seeds:
                dxp = (x - sx + L / 2) % L - L / 2
                dyp = (y - sy + L / 2) % L - L / 2
                if math.hypot(dxp, dyp) < r + sr + 4.0:
                    ok = False
                    break
            if ok:
                crystals.append(dict(kind=1, eps=rng.uniform(0.01, 0.07), q=4, phi0=rng.uniform(0, math.pi / 2)))
                seeds.append((x, y, 0.0, r, len(seeds)))
        out.append(dict(shape=(1, L, L), params=dict(C4_PARAMS, delta=delta), crystals=crystals, seeds=seeds))
    return out


def surrogate_draws(n, size=128, seed=20260101, max_seeds=2):
    """Random single-domain 2D draws for the surrogate's training data, with
    the batched configuration's distributions (parameter set of Sec. 4.3):
    1..max_seeds seeds of radius U[4, 10], angle-form crystals q = 4 with
    theta ~ U[0, pi/2), eps ~ U[0.01, 0.07], Delta ~ U[0.2, 0.6]."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(n):
        ns = rng.randint(1, max_seeds)
        delta = rng.uniform(0.2, 0.6)
        seeds, crystals = [], []
        tries = 0
        while len(seeds) < ns and tries < 1000:
            tries += 1
            r = rng.uniform(4.0, 10.0)
            x, y = rng.uniform(0, size), rng.uniform(0, size)
            if all(math.hypot((x - sx + size / 2) % size - size / 2, (y - sy + size / 2) % size - size / 2) >= r + sr + 4.0
                   for (sx, sy, _, sr, _) in seeds):
                crystals.append(dict(kind=1, eps=rng.uniform(0.01, 0.07), q=4, phi0=rng.uniform(0, math.pi / 2)))
                seeds.append((x, y, 0.0, r, len(seeds)))
        out.append(dict(shape=(1, size, size), params=dict(C4_PARAMS, delta=delta), crystals=crystals, seeds=seeds))
    return out
