"""Hermite tensors, polynomial equilibria, BGK and recursive-regularized (RR) collisions.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sources (arXiv 2504.04465, Appendix A):
  * Hermite tensors: the 2D list printed after Eq. GenEq; in general Grad's recursion
        H^(n+1)_{a b} = xi_b H^(n)_a - theta sum_k delta_{b a_k} H^(n-1)_{a without a_k},
    with theta the reference temperature (c_s^2 for weakly compressible models).
  * Which tensors each lattice keeps: Tab. lattices_hermite (cyclic permutations included).
    D3Q27 is not in the table; its basis is every tensor in which each axis appears at most
    twice (the reading stated in the design notes, R6).
  * Equilibrium (Eq. GenEq):  f_i^eq = w_i sum_n 1/(n! theta^n) H^(n)_i : a^(n)_eq, the
    contraction ':' running over ALL index tuples, so a unique component counts with its
    multinomial multiplicity.  Athermal moments follow Eq. RecursivityEquilibrium,
    a^(n)_eq = rho u...u.  The thermal moments of a Maxwellian of temperature T expanded about
    theta (reading R9, used by the compressible polynomial model) add, for every set of
    disjoint index pairs, a factor (T - theta) delta per pair.
  * RR (Eq. GenRegCollision): f*_i = w_i sum_n 1/(n! c_s^2n) H^(n)_i : (a_eq + (1-1/tau) a_neq),
    with Pi = sum_i H^(2)_i (f_i - f^eq_i) and, for n >= 2, the pair-sum form of the
    recursion of Eq. a1Rec (reading R5):
        a_neq,(a_1..a_n) = sum_{p<q} Pi_{a_p a_q} prod_{k != p,q} u_{a_k}.
    The tests check this form against the six explicit N=4 formulas printed in Eq. a1Rec.
"""
from __future__ import annotations

from functools import lru_cache
from itertools import combinations
from math import factorial

import numpy as np

from .lattices import Lattice


# ----------------------------------------------------------------------------- tensors
def hermite_tensor(xi: np.ndarray, alpha: tuple[int, ...], theta: float) -> np.ndarray:
    """H^(n)_alpha evaluated at every velocity of ``xi`` (shape (Q, D)) -> (Q,).

    Grad's recursion on the last index of ``alpha``.
    """
    xi = np.asarray(xi, dtype=np.float64)
    n = len(alpha)
    if n == 0:
        return np.ones(xi.shape[0])
    head, b = alpha[:-1], alpha[-1]
    out = xi[:, b] * hermite_tensor(xi, head, theta)
    for k, a in enumerate(head):
        if a == b:
            out = out - theta * hermite_tensor(xi, head[:k] + head[k + 1:], theta)
    return out


def counts_to_tuple(counts: tuple[int, ...]) -> tuple[int, ...]:
    """(nx, ny[, nz]) -> sorted index tuple, e.g. (2, 1) -> (0, 0, 1)."""
    out: list[int] = []
    for axis, c in enumerate(counts):
        out += [axis] * c
    return tuple(out)


def multiplicity(counts: tuple[int, ...]) -> int:
    """Number of index tuples that are permutations of the component ``counts``."""
    n = sum(counts)
    m = factorial(n)
    for c in counts:
        m //= factorial(c)
    return m


def _all_counts(D: int, n: int) -> list[tuple[int, ...]]:
    if D == 1:
        return [(n,)]
    out = []
    for c0 in range(n, -1, -1):
        for rest in _all_counts(D - 1, n - c0):
            out.append((c0,) + rest)
    return out


@lru_cache(maxsize=None)
def basis_components(lattice_name: str, D: int) -> tuple[tuple[int, ...], ...]:
    """Unique tensor components kept by each lattice (Tab. lattices_hermite).

    D2Q9: H0, H1, all H2, xxy/xyy, xxyy.  D2Q13/D2Q21: everything up to order 3.
    D2Q37: everything up to order 4.  D3Q27: every axis at most twice (orders 0..6).
    """
    if lattice_name == "D2Q9":
        keep = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (2, 1), (1, 2), (2, 2)]
    elif lattice_name in ("D2Q13", "D2Q21"):
        keep = [c for n in range(4) for c in _all_counts(2, n)]
    elif lattice_name == "D2Q37":
        keep = [c for n in range(5) for c in _all_counts(2, n)]
    elif lattice_name == "D3Q27":
        keep = [c for n in range(7) for c in _all_counts(3, n) if max(c) <= 2]
    else:
        raise ValueError(lattice_name)
    return tuple(keep)


def thermal_basis_components(lattice_name: str, order: int) -> tuple[tuple[int, ...], ...]:
    """All 2D components up to ``order`` (used by the compressible polynomial equilibria)."""
    return tuple(c for n in range(order + 1) for c in _all_counts(2, n))


# ----------------------------------------------------------------------------- moments
def _matchings(positions: tuple[int, ...]):
    """All sets of disjoint pairs (partial matchings) of ``positions``."""
    if len(positions) < 2:
        yield ()
        return
    first, rest = positions[0], positions[1:]
    # first unmatched
    for m in _matchings(rest):
        yield m
    # first matched with one of the rest
    for j, p in enumerate(rest):
        remaining = rest[:j] + rest[j + 1:]
        for m in _matchings(remaining):
            yield ((first, p),) + m


def a_eq(alpha: tuple[int, ...], rho: np.ndarray, u: np.ndarray, dT=None) -> np.ndarray:
    """Equilibrium Hermite moment a^(n)_alpha for every cell.

    rho (n,), u (D, n).  dT = T - theta (n,) or None (athermal: a = rho u...u).
    Thermal moments: sum over partial matchings of the index positions, each pair giving
    dT * delta, each unmatched index giving u.
    """
    if dT is None:
        out = rho.copy()
        for a in alpha:
            out = out * u[a]
        return out
    total = np.zeros_like(rho)
    for m in _matchings(tuple(range(len(alpha)))):
        matched = {p for pair in m for p in pair}
        if any(alpha[p] != alpha[q] for p, q in m):
            continue                       # delta_{a_p a_q} = 0
        term = rho * dT ** len(m) if m else rho.copy()
        for k, a in enumerate(alpha):
            if k not in matched:
                term = term * u[a]
        total = total + term
    return total


def a_neq(alpha: tuple[int, ...], Pi: dict, u: np.ndarray) -> np.ndarray:
    """Non-equilibrium Hermite moment by the pair-sum closed form (reading R5)."""
    n = len(alpha)
    if n < 2:
        return np.zeros_like(u[0])
    total = np.zeros_like(u[0])
    for p, q in combinations(range(n), 2):
        term = Pi[tuple(sorted((alpha[p], alpha[q])))].copy()
        for k in range(n):
            if k != p and k != q:
                term = term * u[alpha[k]]
        total = total + term
    return total


def macroscopic(lat: Lattice, f: np.ndarray):
    """rho = sum f, u = sum xi f / rho  (f: (Q, n))."""
    rho = f.sum(axis=0)
    u = (lat.xi.T.astype(np.float64) @ f) / rho
    return rho, u


def expand(lat: Lattice, comps, theta: float, moments) -> np.ndarray:
    """w_i sum_n 1/(n! theta^n) sum_{all tuples} H^(n)_{i,alpha} A_alpha  -> (Q, n).

    ``moments(alpha)`` returns A_alpha for every cell.
    """
    acc = None
    for c in comps:
        alpha = counts_to_tuple(c)
        n = len(alpha)
        H = hermite_tensor(lat.xi, alpha, theta)                     # (Q,)
        coef = multiplicity(c) / (factorial(n) * theta ** n)
        term = coef * H[:, None] * moments(alpha)[None, :]
        acc = term if acc is None else acc + term
    return lat.w[:, None] * acc


def feq_athermal(lat: Lattice, rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Eq. GenEq with the lattice's basis and T0 = c_s^2 (weakly compressible models)."""
    comps = basis_components(lat.name, lat.D)
    return expand(lat, comps, lat.cs2, lambda al: a_eq(al, rho, u))


def feq_thermal(lat: Lattice, rho: np.ndarray, u: np.ndarray, T: np.ndarray, order: int) -> np.ndarray:
    """Thermal Hermite equilibrium about theta = c_s^2, all components up to ``order`` (R9)."""
    comps = thermal_basis_components(lat.name, order)
    dT = T - lat.cs2
    return expand(lat, comps, lat.cs2, lambda al: a_eq(al, rho, u, dT))


def pi_neq(lat: Lattice, f: np.ndarray, feq: np.ndarray) -> dict:
    """Pi_ab = sum_i H^(2)_{i,ab} (f_i - f^eq_i) for a <= b."""
    fneq = f - feq
    Pi = {}
    for a in range(lat.D):
        for b in range(a, lat.D):
            H2 = hermite_tensor(lat.xi, (a, b), lat.cs2)
            Pi[(a, b)] = H2 @ fneq
    return Pi


def collide_bgk(f: np.ndarray, feq: np.ndarray, tau) -> np.ndarray:
    """Eq. CollisionStep: f* = f - (f - f^eq)/tau."""
    return f - (f - feq) / tau


def collide_rr(lat: Lattice, f: np.ndarray, tau, trace_eq: bool = False) -> np.ndarray:
    """Recursive-regularized collision, Eq. GenRegCollision.

    trace_eq: equilibrate the trace of the second-order moments (Appendix A, after Eq. a1Rec;
    the bulk relaxation time set to one): Pi is replaced by its deviatoric part
    Pi - (tr Pi / D) I before the recursion, so no trace survives the collision (reading R35)."""
    rho, u = macroscopic(lat, f)
    feq = feq_athermal(lat, rho, u)
    Pi = pi_neq(lat, f, feq)
    if trace_eq:
        tr = sum(Pi[(a, a)] for a in range(lat.D)) / lat.D
        Pi = {k: (v - tr if k[0] == k[1] else v) for k, v in Pi.items()}
    comps = basis_components(lat.name, lat.D)
    omega = 1.0 - 1.0 / np.asarray(tau, dtype=np.float64)
    return expand(lat, comps, lat.cs2,
                  lambda al: a_eq(al, rho, u) + omega * a_neq(al, Pi, u))


def trt_omega_minus(tau_plus: float, magic: float) -> float:
    """Relaxation rate of the antisymmetric part of the two-relaxation-time collision from the
    'magic' combination Lambda = (tau+ - 1/2)(tau- - 1/2) (reading R36)."""
    if tau_plus <= 0.5:
        raise ValueError("the two-relaxation-time collision needs tau+ > 1/2 (a positive viscosity)")
    return 1.0 / (magic / (tau_plus - 0.5) + 0.5)


def collide_trt(lat: Lattice, f: np.ndarray, feq: np.ndarray, tau, magic: float) -> np.ndarray:
    """Two-relaxation-time collision: the parts of f - f_eq even and odd under xi -> -xi relax
    with 1/tau+ (tau+ = tau, the viscosity) and with the rate of ``trt_omega_minus``."""
    opp = lat.opp
    wp = 1.0 / tau
    wm = trt_omega_minus(tau, magic)
    d = f - feq
    even = 0.5 * (d + d[opp])
    odd = 0.5 * (d - d[opp])
    return f - wp * even - wm * odd


def collide_weak(lat: Lattice, f: np.ndarray, tau, model: str, trace_eq: bool = False,
                 magic: float = 0.25) -> np.ndarray:
    """Weakly compressible collision: model 'bgk', 'trt' or 'rr' (same equilibrium, Sec. A.2)."""
    if model == "rr":
        return collide_rr(lat, f, tau, trace_eq)
    rho, u = macroscopic(lat, f)
    if model == "trt":
        return collide_trt(lat, f, feq_athermal(lat, rho, u), tau, magic)
    return collide_bgk(f, feq_athermal(lat, rho, u), tau)
