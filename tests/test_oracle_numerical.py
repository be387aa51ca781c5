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


@pytest.mark.parametrize("name,T0", [("D2Q13", 0.35), ("D2Q21", 0.65), ("D2Q21", 0.9), ("D2Q37", 1.0)])
def test_newton_satisfies_printed_constraints(name, T0):
    lat = L.LATTICES[name]
    n = 64
    u = RNG.uniform(-0.6, 0.6, size=(2, n)) * np.sqrt(T0)
    T = T0 * RNG.uniform(0.7, 1.4, size=n)
    lam0 = nm.poly_guess(lat, u, T, 4 if lat.Q == 37 else 3)
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


def test_cholesky_solve_matches_library_and_flags_singular():
    rng = np.random.default_rng(21)
    B = rng.standard_normal((40, 8, 8))
    A = B @ np.transpose(B, (0, 2, 1)) + 0.1 * np.eye(8)
    b = rng.standard_normal((40, 8))
    x = nm.cholesky_solve(A, b)
    ref = np.linalg.solve(A, b[:, :, None])[:, :, 0]
    assert np.abs(x - ref).max() < 1e-10 * np.abs(ref).max()
    S = A[:2].copy()
    S[0, 3, :] = S[0, :, 3] = 0.0            # singular (zero row and column)
    S[1, 5, 5] = -1.0                        # not positive definite
    assert np.isnan(nm.cholesky_solve(S, b[:2])).all()


def test_polynomial_guess_is_the_weighted_fit_where_it_helps():
    lat = L.LATTICES["D2Q21"]
    from oracle import hermite as hm
    u = np.array([[0.2], [0.1]])
    T = np.array([0.7])
    g = nm.poly_guess(lat, u, T, 3)[:, 0]
    # the same weighted least-squares problem through the library's lstsq
    fp = hm.feq_thermal(lat, np.ones(1), u, T, 3)[:, 0]
    pos = fp > 0
    M = nm.moment_basis(lat)
    sw = np.sqrt(lat.w[pos])
    ref = np.linalg.lstsq(M[:, pos].T * sw[:, None], (-1.0 - np.log(fp[pos])) * sw, rcond=None)[0]
    assert np.abs(g - ref).max() < 1e-10


def test_polynomial_guess_falls_back_to_zero_at_high_mach():
    lat = L.LATTICES["D2Q21"]
    from oracle import hermite as hm
    u = np.array([[1.43], [0.0]])            # Mach 1.5 at T = 0.65 (gamma 1.4)
    T = np.array([0.65])
    g = nm.poly_guess(lat, u, T, 3)
    assert np.array_equal(g, np.zeros((8, 1)))
    # there the fit itself is farther from the root than lambda = 0
    fp = hm.feq_thermal(lat, np.ones(1), u, T, 3)[:, 0]
    pos = fp > 0
    M = nm.moment_basis(lat)
    sw = np.sqrt(lat.w[pos])
    fit = np.linalg.lstsq(M[:, pos].T * sw[:, None], (-1.0 - np.log(fp[pos])) * sw, rcond=None)[0]
    tgt = nm.mb_targets(u, T)
    Gf, _ = nm.residual(M, fit[:, None], tgt)
    G0, _ = nm.residual(M, np.zeros((8, 1)), tgt)
    assert (Gf ** 2).sum() > (G0 ** 2).sum()
    lam, e, it, conv = nm.newton(lat, u, T, g, 1e-12, 50)
    assert conv.all()


def test_newton_stops_without_error_at_an_unreachable_state():
    lat = L.LATTICES["D2Q21"]
    u = np.array([[2.0, 0.1], [0.0, 0.0]])   # |u| = 2: beyond the lattice (exp underflow)
    T = np.array([0.65, 0.65])
    lam, e, it, conv = nm.newton(lat, u, T, np.zeros((8, 2)), 1e-12, 50)
    assert not conv[0] and conv[1]
    assert it[0] < 50
    assert np.isfinite(e).all() and np.isfinite(lam).all()
