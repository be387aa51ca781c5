"""Pins of the max-entropy Newton solver against the printed constraints (Eqs. G0..G3yaa)."""
import numpy as np
import pytest

from oracle import lattices as L
from oracle import numerical as nm

RNG = np.random.default_rng(1504)


def _printed_constraints(lat, f, rho, ux, uy, T):
    """Eqs. G0_8mom .. G3yaa_8mom written out, with 2E = ux^2 + uy^2 + 2T."""
    x = lat.xi[:, 0].astype(float)[:, None]
    y = lat.xi[:, 1].astype(float)[:, None]
    E = 0.5 * (ux ** 2 + uy ** 2 + 2 * T)
    return np.stack([
        f.sum(0) - rho,
        (f * x).sum(0) - rho * ux,
        (f * y).sum(0) - rho * uy,
        (f * x * x).sum(0) - rho * (ux ** 2 + T),
        (f * x * y).sum(0) - rho * ux * uy,
        (f * y * y).sum(0) - rho * (uy ** 2 + T),
        (f * x * (x * x + y * y)).sum(0) - 2 * rho * ux * (E + T),
        (f * y * (x * x + y * y)).sum(0) - 2 * rho * uy * (E + T),
    ])


@pytest.mark.parametrize("name,T0", [("D2Q21", 0.65), ("D2Q21", 0.9), ("D2Q37", 1.0)])
def test_newton_satisfies_printed_constraints(name, T0):
    lat = L.LATTICES[name]
    n = 64
    u = RNG.uniform(-0.6, 0.6, size=(2, n)) * np.sqrt(T0)
    T = T0 * RNG.uniform(0.7, 1.4, size=n)
    lam0 = nm.poly_guess(lat, u, T, 3 if lat.Q == 21 else 4)
    lam, e, it, conv = nm.newton(lat, u, T, lam0, tol=1e-12)
    assert conv.all()
    for rho in (1.0, 7.3):                       # rho-independence of lambda (a = rho)
        G = _printed_constraints(lat, rho * e, rho, u[0], u[1], T)
        assert np.abs(G).max() < 1e-12 * rho * 10
    assert it.max() <= 12


def test_symmetry_at_rest():
    lat = L.D2Q21
    n = 5
    u = np.zeros((2, n))
    T = np.linspace(0.6, 1.0, n)
    lam, e, it, conv = nm.newton(lat, u, T, np.zeros((8, n)))
    assert conv.all()
    assert np.abs(lam[[1, 2, 4, 6, 7]]).max() < 1e-11          # x, y, xy, x|xi|^2, y|xi|^2
    assert np.abs(lam[3] - lam[5]).max() < 1e-11               # xx == yy


def test_warm_start_takes_fewer_iterations():
    lat = L.D2Q21
    n = 100
    u = RNG.uniform(-0.3, 0.3, size=(2, n))
    T = 0.9 * RNG.uniform(0.8, 1.2, size=n)
    _, _, it_zero, c0 = nm.newton(lat, u, T, np.zeros((8, n)))
    lam, _, _, _ = nm.newton(lat, u, T, nm.poly_guess(lat, u, T, 3))
    # a slightly perturbed state, warm-started from the neighbouring solution
    lam2, _, it_warm, c1 = nm.newton(lat, u * 1.001, T * 1.001, lam)
    assert c0.all() and c1.all()
    assert it_zero.mean() >= 5 and it_warm.mean() <= 3


def test_line_search_never_increases_residual():
    lat = L.D2Q21
    n = 20
    u = RNG.uniform(-0.8, 0.8, size=(2, n))
    T = RNG.uniform(0.5, 1.5, size=n)
    M = nm.moment_basis(lat)
    tgt = nm.mb_targets(u, T)
    lam = np.zeros((8, n))
    prev = np.linalg.norm(nm.residual(M, lam, tgt)[0], axis=0)
    for k in range(1, 8):
        lam_k, _, it, _ = nm.newton(lat, u, T, np.zeros((8, n)), tol=1e-30, max_iter=k)
        cur = np.linalg.norm(nm.residual(M, lam_k, tgt)[0], axis=0)
        assert np.all(cur <= prev * (1 + 1e-12) + 1e-300)
        prev = cur
