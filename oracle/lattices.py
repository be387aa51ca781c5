"""Velocity sets used by the method (Appendix A, Tab. lattices_structure and Fig. lattices).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Each lattice is built from its symmetry groups exactly as the table lists them: a group
(a, b) contributes every signed permutation of (a, b).  Weights are the printed fractions
for D2Q9, D2Q13 and D2Q21.  For D2Q37 the table prints 15 decimals only, so the weights and
c_s^2 are re-derived here in FP64 by solving the lattice's isotropy conditions (moments of the
weight function equal those of a Gaussian up to 8th order) with Newton's method, started from
the printed values; the tests check the result against the table to 1e-14.  D3Q27 is not in
the table: it is the tensor product of the 1D three-velocity lattice (weights 2/3, 1/6, 1/6,
c_s^2 = 1/3), which the tests pin by its isotropy.
"""
from __future__ import annotations

from dataclasses import dataclass
from fractions import Fraction
from itertools import product

import numpy as np


@dataclass(frozen=True)
class Lattice:
    name: str
    D: int
    xi: np.ndarray      # (Q, D) integer velocities
    w: np.ndarray       # (Q,) weights, FP64
    cs2: float          # lattice constant c_s^2

    @property
    def Q(self) -> int:
        return self.xi.shape[0]

    @property
    def reach(self) -> int:
        """Largest |xi|_inf: the number of ghost/boundary layers the lattice needs (Sec. 3.2)."""
        return int(np.abs(self.xi).max())

    @property
    def opp(self) -> np.ndarray:
        """Index of -xi_i for every i (used by bounce-back)."""
        idx = {tuple(v): i for i, v in enumerate(self.xi)}
        return np.array([idx[tuple(-v)] for v in self.xi], dtype=np.int64)


def _signed_perms_2d(a: int, b: int) -> list[tuple[int, int]]:
    out = set()
    for p, q in ((a, b), (b, a)):
        for sp in (1, -1):
            for sq in (1, -1):
                out.add((sp * p, sq * q))
    return sorted(out)


def _lattice_2d(name: str, groups: list[tuple[int, int]], weights: list[float], cs2: float) -> Lattice:
    xi, w = [], []
    for g, wg in zip(groups, weights):
        for v in _signed_perms_2d(*g):
            xi.append(v)
            w.append(wg)
    return Lattice(name, 2, np.array(xi, dtype=np.int64), np.array(w, dtype=np.float64), float(cs2))


D2Q9 = _lattice_2d("D2Q9", [(0, 0), (1, 0), (1, 1)],
                   [4 / 9, 1 / 9, 1 / 36], 1 / 3)
D2Q13 = _lattice_2d("D2Q13", [(0, 0), (1, 0), (1, 1), (2, 0)],
                    [36 / 96, 8 / 96, 6 / 96, 1 / 96], 1 / 2)
D2Q21 = _lattice_2d("D2Q21", [(0, 0), (1, 0), (1, 1), (2, 0), (2, 2), (3, 0)],
                    [91 / 324, 1 / 12, 2 / 27, 7 / 360, 1 / 432, 1 / 1620], 2 / 3)

# D2Q37 groups in the order of the table; the printed weights seed the Newton solve below.
D2Q37_GROUPS = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 1)]
D2Q37_PRINTED_W = [0.233150669132352, 0.107306091542219, 0.057667859888794, 0.014208216158450,
                   0.005353049000513, 0.001011937592673, 0.000245301027757, 0.000283414252994]
D2Q37_PRINTED_CS2 = 0.697953322019683


def _d2q37_weights() -> tuple[list[float], float]:
    """Solve the 9 isotropy conditions for the 8 group weights and theta = c_s^2.

    Conditions (Gaussian moments of a 2D isotropic distribution with variance theta):
        sum w = 1, <x^2> = th, <x^4> = 3 th^2, <x^2 y^2> = th^2, <x^6> = 15 th^3,
        <x^4 y^2> = 3 th^3, <x^8> = 105 th^4, <x^6 y^2> = 15 th^4, <x^4 y^4> = 9 th^4.
    """
    orbits = [_signed_perms_2d(*g) for g in D2Q37_GROUPS]

    def row(px, py):
        return np.array([sum(float(x) ** px * float(y) ** py for x, y in o) for o in orbits])

    # (px, py, coefficient c, power k): sum_g w_g * row = c * theta^k
    conds = [(0, 0, 1, 0), (2, 0, 1, 1), (4, 0, 3, 2), (2, 2, 1, 2), (6, 0, 15, 3),
             (4, 2, 3, 3), (8, 0, 105, 4), (6, 2, 15, 4), (4, 4, 9, 4)]
    A = np.array([row(px, py) for px, py, _, _ in conds])
    z = np.array(D2Q37_PRINTED_W + [D2Q37_PRINTED_CS2], dtype=np.float64)
    for _ in range(50):
        w, th = z[:8], z[8]
        F = A @ w - np.array([c * th ** k for _, _, c, k in conds])
        J = np.zeros((9, 9))
        J[:, :8] = A
        J[:, 8] = [-(c * k * th ** (k - 1)) if k > 0 else 0.0 for _, _, c, k in conds]
        dz = np.linalg.solve(J, F)
        z = z - dz
        if np.abs(dz).max() < 1e-17:
            break
    return list(z[:8]), float(z[8])


_w37, _cs2_37 = _d2q37_weights()
D2Q37 = _lattice_2d("D2Q37", D2Q37_GROUPS, _w37, _cs2_37)


def _d3q27() -> Lattice:
    w1 = {-1: 1 / 6, 0: 2 / 3, 1: 1 / 6}
    xi, w = [], []
    for v in product((-1, 0, 1), repeat=3):
        xi.append(v)
        w.append(w1[v[0]] * w1[v[1]] * w1[v[2]])
    # order: rest first, then by |xi|^2, then lexicographic -- a fixed, documented order
    order = sorted(range(27), key=lambda i: (sum(c * c for c in xi[i]), xi[i]))
    return Lattice("D3Q27", 3, np.array([xi[i] for i in order], dtype=np.int64),
                   np.array([w[i] for i in order], dtype=np.float64), 1 / 3)


D3Q27 = _d3q27()

LATTICES = {lat.name: lat for lat in (D2Q9, D2Q13, D2Q21, D2Q37, D3Q27)}

# exact fractions of the printed table (used by the pins)
PRINTED_FRACTIONS = {
    "D2Q9": ([Fraction(4, 9), Fraction(1, 9), Fraction(1, 36)], Fraction(1, 3)),
    "D2Q13": ([Fraction(36, 96), Fraction(8, 96), Fraction(6, 96), Fraction(1, 96)], Fraction(1, 2)),
    "D2Q21": ([Fraction(91, 324), Fraction(1, 12), Fraction(2, 27), Fraction(7, 360), Fraction(1, 432),
               Fraction(1, 1620)], Fraction(2, 3)),
}
PRINTED_GROUPS = {
    "D2Q9": [(0, 0), (1, 0), (1, 1)],
    "D2Q13": [(0, 0), (1, 0), (1, 1), (2, 0)],
    "D2Q21": [(0, 0), (1, 0), (1, 1), (2, 0), (2, 2), (3, 0)],
    "D2Q37": D2Q37_GROUPS,
}
