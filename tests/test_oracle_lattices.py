"""Pins of the oracle's velocity sets: printed weights (Tab. lattices_structure) and isotropy."""
from fractions import Fraction
from itertools import product

import numpy as np
import pytest

from oracle import lattices as L


def _moment(lat, px, py, pz=0):
    xi = lat.xi.astype(np.float64)
    m = lat.w * xi[:, 0] ** px * xi[:, 1] ** py
    if lat.D == 3:
        m = m * xi[:, 2] ** pz
    return m.sum()


@pytest.mark.parametrize("name", ["D2Q9", "D2Q13", "D2Q21"])
def test_printed_fractions(name):
    lat = L.LATTICES[name]
    weights, cs2 = L.PRINTED_FRACTIONS[name]
    groups = L.PRINTED_GROUPS[name]
    assert lat.cs2 == float(cs2)
    total = Fraction(0)
    for g, w in zip(groups, weights):
        members = [i for i, v in enumerate(lat.xi) if sorted(map(abs, v)) == sorted(g)]
        assert len(members) in (1, 4, 8)
        for i in members:
            assert lat.w[i] == float(w)
        total += w * len(members)
    assert total == 1  # exact


@pytest.mark.parametrize("name,order", [("D2Q9", 4), ("D2Q13", 4), ("D2Q21", 6), ("D2Q37", 8)])
def test_isotropy_2d(name, order):
    lat = L.LATTICES[name]
    th = lat.cs2
    # Gaussian moments <x^a y^b> = (a-1)!! (b-1)!! th^((a+b)/2) for even a, b
    def dfact(n):
        return 1 if n <= 0 else n * dfact(n - 2)
    for a in range(0, order + 1, 2):
        for b in range(0, order + 1 - a, 2):
            expect = dfact(a - 1) * dfact(b - 1) * th ** ((a + b) // 2)
            assert abs(_moment(lat, a, b) - expect) < 1e-13, (a, b)
    # odd moments vanish
    assert abs(_moment(lat, 1, 0)) < 1e-15 and abs(_moment(lat, 3, 1)) < 1e-15


def test_d2q37_rederived_against_table():
    lat = L.D2Q37
    assert abs(lat.cs2 - L.D2Q37_PRINTED_CS2) < 1e-14
    for g, w in zip(L.D2Q37_GROUPS, L.D2Q37_PRINTED_W):
        members = [i for i, v in enumerate(lat.xi) if sorted(map(abs, v)) == sorted(g)]
        assert abs(lat.w[members[0]] - w) < 1e-14
        assert np.all(lat.w[members] == lat.w[members[0]])
    assert abs(lat.w.sum() - 1.0) < 1e-15
    assert lat.Q == 37


def test_d3q27_textbook():
    lat = L.D3Q27
    expect = {0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216}
    for v, w in zip(lat.xi, lat.w):
        assert w == pytest.approx(expect[int(np.abs(v).sum())], abs=1e-17)
    th = lat.cs2
    assert abs(_moment(lat, 0, 0, 0) - 1) < 1e-15
    assert abs(_moment(lat, 2, 0, 0) - th) < 1e-15
    assert abs(_moment(lat, 4, 0, 0) - th ** 2) > 0.01          # D1Q3: not 4th-order in 1 axis
    assert abs(_moment(lat, 2, 2, 0) - th ** 2) < 1e-15
    assert abs(_moment(lat, 2, 2, 2) - th ** 3) < 1e-15


@pytest.mark.parametrize("name", list(L.LATTICES))
def test_opposites_and_reach(name):
    lat = L.LATTICES[name]
    assert np.all(lat.xi[lat.opp] == -lat.xi)
    assert lat.reach == {"D2Q9": 1, "D2Q13": 2, "D2Q21": 3, "D2Q37": 3, "D3Q27": 1}[name]
    assert len({tuple(v) for v in lat.xi}) == lat.Q
