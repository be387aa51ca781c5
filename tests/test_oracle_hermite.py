"""Pins of the Hermite machinery against the formulas printed in Appendix A, and invariants."""
import numpy as np
import pytest

from oracle import hermite as hm
from oracle import lattices as L

RNG = np.random.default_rng(2504)


def test_hermite_tensors_match_printed_2d():
    # Appendix A lists the 2D Hermite tensors up to fourth order explicitly
    lat = L.D2Q37
    x = lat.xi[:, 0].astype(float)
    y = lat.xi[:, 1].astype(float)
    c = 0.7
    printed = {
        (0, 0): x * x - c, (0, 1): x * y,
        (0, 0, 0): (x * x - 3 * c) * x, (0, 0, 1): (x * x - c) * y,
        (0, 0, 0, 0): x ** 4 - 6 * c * x * x + 3 * c * c,
        (0, 0, 0, 1): (x * x - 3 * c) * x * y,
        (0, 0, 1, 1): (x * x - c) * (y * y - c),
    }
    for alpha, ref in printed.items():
        assert np.allclose(hm.hermite_tensor(lat.xi, alpha, c), ref, atol=1e-13, rtol=0)
        # symmetric in the order of the indices
        assert np.allclose(hm.hermite_tensor(lat.xi, alpha[::-1], c), ref, atol=1e-13, rtol=0)


def test_basis_sizes_follow_table():
    assert len(hm.basis_components("D2Q9", 2)) == 9
    assert len(hm.basis_components("D2Q21", 2)) == 10
    assert len(hm.basis_components("D2Q37", 2)) == 15
    assert len(hm.basis_components("D3Q27", 3)) == 27
    # D2Q9 keeps xxy, xyy, xxyy but not xxx, xxxx, xxxy
    comps = set(hm.basis_components("D2Q9", 2))
    assert {(2, 1), (1, 2), (2, 2)} <= comps and not {(3, 0), (4, 0), (3, 1)} & comps


def test_rr_pair_sum_reproduces_printed_n4_formulas():
    """Eq. a1Rec prints the N=4 non-equilibrium moments of the recursion explicitly."""
    n = 50
    u = RNG.normal(size=(2, n)) * 0.2
    Pi = {(0, 0): RNG.normal(size=n), (0, 1): RNG.normal(size=n), (1, 1): RNG.normal(size=n)}
    ux, uy = u
    a2xx, a2xy, a2yy = Pi[(0, 0)], Pi[(0, 1)], Pi[(1, 1)]
    a3xxx = 3 * ux * a2xx
    a3xxy = 2 * ux * a2xy + uy * a2xx
    a3yyx = 2 * uy * a2xy + ux * a2yy
    a4xxxx = 4 * ux * a3xxx - 6 * ux ** 2 * a2xx
    a4xxxy = (3 * ux * a3xxy + uy * a3xxx) - 3 * ux ** 2 * a2xy - 3 * ux * uy * a2xx
    a4xxyy = 2 * (ux * a3yyx + uy * a3xxy) - ux ** 2 * a2yy - uy ** 2 * a2xx - 4 * ux * uy * a2xy
    got = {al: hm.a_neq(al, Pi, u) for al in [(0, 0), (0, 1), (0, 0, 0), (0, 0, 1), (0, 0, 0, 0),
                                              (0, 0, 0, 1), (0, 0, 1, 1)]}
    for al, ref in [((0, 0), a2xx), ((0, 1), a2xy), ((0, 0, 0), a3xxx), ((0, 0, 1), a3xxy),
                    ((0, 0, 0, 0), a4xxxx), ((0, 0, 0, 1), a4xxxy), ((0, 0, 1, 1), a4xxyy)]:
        assert np.allclose(got[al], ref, atol=1e-13, rtol=1e-13), al


def test_thermal_moments_are_gaussian_hermite_coefficients():
    # 1D closed forms: int N(u,T) (x^2 - th) = u^2 + T - th;  (x^3 - 3 th x) -> u^3 + 3u(T - th);
    # (x^4 - 6 th x^2 + 3 th^2) -> u^4 + 6 u^2 (T - th) + 3 (T - th)^2
    rho = np.array([1.3])
    u = np.array([[0.37], [0.0]])
    T, th = 0.9, 0.7
    dT = np.array([T - th])
    assert hm.a_eq((0, 0), rho, u, dT)[0] == pytest.approx(1.3 * (0.37 ** 2 + T - th))
    assert hm.a_eq((0, 0, 0), rho, u, dT)[0] == pytest.approx(1.3 * (0.37 ** 3 + 3 * 0.37 * (T - th)))
    assert hm.a_eq((0, 0, 0, 0), rho, u, dT)[0] == pytest.approx(
        1.3 * (0.37 ** 4 + 6 * 0.37 ** 2 * (T - th) + 3 * (T - th) ** 2))
    assert hm.a_eq((0, 1), rho, u, dT)[0] == pytest.approx(0.0)       # u_y = 0, no delta_xy


@pytest.mark.parametrize("name", ["D2Q9", "D3Q27", "D2Q13", "D2Q21", "D2Q37"])
def test_athermal_equilibrium_moments(name):
    lat = L.LATTICES[name]
    n = 40
    rho = 1 + 0.1 * RNG.random(n)
    u = 0.1 * RNG.normal(size=(lat.D, n))
    feq = hm.feq_athermal(lat, rho, u) if name in ("D2Q9", "D3Q27") else hm.feq_thermal(lat, rho, u, np.full(n, lat.cs2), 3)
    xi = lat.xi.astype(float)
    assert np.allclose(feq.sum(0), rho, atol=1e-14, rtol=0)
    assert np.allclose(xi.T @ feq, rho * u, atol=1e-14, rtol=0)
    for a in range(lat.D):
        for b in range(lat.D):
            ref = rho * (u[a] * u[b] + (lat.cs2 if a == b else 0.0))
            assert np.allclose((xi[:, a] * xi[:, b]) @ feq, ref, atol=1e-14, rtol=0)


def test_thermal_equilibrium_moments_d2q37():
    lat = L.D2Q37
    n = 30
    rho = 1 + 0.2 * RNG.random(n)
    u = 0.2 * RNG.normal(size=(2, n))
    T = lat.cs2 * (0.8 + 0.4 * RNG.random(n))
    feq = hm.feq_thermal(lat, rho, u, T, 4)
    xi = lat.xi.astype(float)
    u2 = (u ** 2).sum(0)
    assert np.allclose(feq.sum(0), rho, atol=1e-14, rtol=0)
    assert np.allclose(xi.T @ feq, rho * u, atol=1e-14, rtol=0)
    assert np.allclose((xi[:, 0] ** 2) @ feq, rho * (u[0] ** 2 + T), atol=1e-13, rtol=0)
    assert np.allclose((xi[:, 0] * xi[:, 1]) @ feq, rho * u[0] * u[1], atol=1e-13, rtol=0)
    r2 = (xi ** 2).sum(1)
    # contracted third moment: rho u_x (|u|^2 + (D+2) T)
    assert np.allclose((xi[:, 0] * r2) @ feq, rho * u[0] * (u2 + 4 * T), atol=1e-12, rtol=0)


@pytest.mark.parametrize("name", ["D2Q9", "D3Q27", "D2Q13", "D2Q21"])
def test_rr_invariants(name):
    lat = L.LATTICES[name]
    n = 25
    rho = 1 + 0.05 * RNG.random(n)
    u = 0.05 * RNG.normal(size=(lat.D, n))
    f = hm.feq_athermal(lat, rho, u) * (1 + 0.02 * RNG.normal(size=(lat.Q, n)))
    tau = 0.7
    fs = hm.collide_rr(lat, f, tau)
    r0, u0 = hm.macroscopic(lat, f)
    r1, u1 = hm.macroscopic(lat, fs)
    assert np.allclose(r1, r0, atol=1e-14, rtol=0)
    assert np.allclose(r1 * u1, r0 * u0, atol=1e-15, rtol=0)
    # Pi* = (1 - 1/tau) Pi
    feq = hm.feq_athermal(lat, r0, u0)
    P0 = hm.pi_neq(lat, f, feq)
    P1 = hm.pi_neq(lat, fs, feq)
    for k in P0:
        assert np.allclose(P1[k], (1 - 1 / tau) * P0[k], atol=1e-15, rtol=0)
    # tau = 1: post-collision state is the equilibrium
    assert np.allclose(hm.collide_rr(lat, f, 1.0), feq, atol=1e-15, rtol=0)
    # BGK at tau = 1 as well
    assert np.allclose(hm.collide_weak(lat, f, 1.0, "bgk"), feq, atol=1e-15, rtol=0)


def test_d2q21_athermal_equilibrium_is_thermal_at_cs2():
    """On D2Q21 the weakly compressible equilibrium (every component to order 3, T0 = c_s^2) is
    the thermal 3rd-order expansion at T = c_s^2, and its contracted third moment is the
    Maxwellian's rho u_x (|u|^2 + (D + 2) c_s^2)."""
    lat = L.D2Q21
    n = 30
    rho = 1 + 0.1 * RNG.random(n)
    u = 0.1 * RNG.normal(size=(2, n))
    feq = hm.feq_athermal(lat, rho, u)
    assert np.allclose(feq, hm.feq_thermal(lat, rho, u, np.full(n, lat.cs2), 3), atol=1e-15, rtol=0)
    xi = lat.xi.astype(float)
    r2 = (xi ** 2).sum(1)
    assert np.allclose((xi[:, 0] * r2) @ feq, rho * u[0] * ((u ** 2).sum(0) + 4 * lat.cs2), atol=1e-13, rtol=0)
