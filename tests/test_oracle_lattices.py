"""Pins of the oracle's lattice tables (Sec. 3.3, Table 1).

Table 1 and the listed displacement vectors are compared entry by entry with
tests/golden/lattices_table1.json; every lattice is checked for the moment
identities the schemes rely on (Sec. 3.1: sum w = 1, sum w e = 0,
sum w e e = e^2 I; Sec. 4.2 relies on the same second moment), and the
phase-field lattices for fourth-order isotropy, exact in rationals.
"""
import json
import os
from fractions import Fraction
from itertools import product

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "lattices_table1.json")))


def frac(x):
    return Fraction(x).limit_denominator(1000)


def test_table1_values(orc):
    O = orc
    cases = [("D2Q9", O.D2Q9_D2Q5, 0), ("D2Q5", O.D2Q9_D2Q5, 1),
             ("D3Q15", O.D3Q15_D3Q7, 0), ("D3Q7", O.D3Q15_D3Q7, 1)]
    for name, lat, which in cases:
        ref = GOLD[name]
        D, e, w, e2 = O.lattice(lat, which)
        assert frac(e2) == Fraction(*ref["e2"]), name
        assert frac(w[0]) == Fraction(*ref["w0"]), name
        assert np.array_equal(e[:, :D], np.array(ref["e"])), name
        for i in range(1, len(w)):
            kind = "w_axis" if np.abs(e[i]).sum() == 1 else "w_diag"
            assert frac(w[i]) == Fraction(*ref[kind]), (name, i)


@pytest.mark.parametrize("lat", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("which", [0, 1])
def test_moments(orc, lat, which):
    D, e, w, e2 = orc.lattice(lat, which)
    W = [frac(x) for x in w]
    # weights are the exact rationals they print as
    assert all(abs(float(Wi) - wi) < 1e-16 for Wi, wi in zip(W, w))
    assert sum(W) == 1
    for a in range(3):
        assert sum(Wi * int(ei[a]) for Wi, ei in zip(W, e)) == 0
        for b in range(3):
            m2 = sum(Wi * int(ei[a]) * int(ei[b]) for Wi, ei in zip(W, e))
            want = frac(e2) if (a == b and a < D) else 0
            assert m2 == want, (lat, which, a, b)
    # every direction has its opposite (needed by streaming on a periodic box)
    s = {tuple(x) for x in e}
    assert all(tuple(-x) in s for x in e)


@pytest.mark.parametrize("lat", [0, 1, 2, 3])
def test_fourth_order_isotropy(orc, lat):
    """sum w e_a e_b e_c e_d = e^4 (d_ab d_cd + d_ac d_bd + d_ad d_bc), e^4 = (e^2)^2;
    this is what makes the directional-derivative gradient isotropic."""
    D, e, w, e2 = orc.lattice(lat, 0)
    W = [frac(x) for x in w]
    e4 = frac(e2) ** 2
    d = lambda i, j: 1 if i == j else 0
    for a, b, c, dd in product(range(D), repeat=4):
        m4 = sum(Wi * int(ei[a]) * int(ei[b]) * int(ei[c]) * int(ei[dd]) for Wi, ei in zip(W, e))
        assert m4 == e4 * (d(a, b) * d(c, dd) + d(a, c) * d(b, dd) + d(a, dd) * d(b, c))


@pytest.mark.parametrize("lat3", [1, 2, 3])
def test_3d_lattices_project_onto_d2q9(orc, lat3):
    """Summing the D3Q15/19/27 weights over e_z gives the D2Q9 weights."""
    _, e9, w9, _ = orc.lattice(0, 0)
    _, e, w, _ = orc.lattice(lat3, 0)
    acc = {}
    for ei, wi in zip(e, w):
        acc[(int(ei[0]), int(ei[1]))] = acc.get((int(ei[0]), int(ei[1])), 0) + frac(wi)
    for ei, wi in zip(e9, w9):
        assert acc[(int(ei[0]), int(ei[1]))] == frac(wi)
