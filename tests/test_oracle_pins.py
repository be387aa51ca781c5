"""Pins of three oracle functions against the paper's definitions and published data.

* The kinetic shock sensor (Appendix A, Eqs. DeltaAvg and shock_function; reading R10 for
  eps < 0.01 and for vanishing f_eq): a threshold table and hand-computed sensor values.
* The boundary pass (Appendix A.3): one pass on hand-set populations checks, cell by cell,
  which cells take an equilibrium Dirichlet value (imposed or extrapolated density), which
  copy their interior partner (Neumann), and which face wins at a corner (reading R12).
* The NACA 0012 solid (reading R20): the half-thickness of the level-0 mask at the stations of
  the published table of ordinates (NACA Report 824, Abbott, von Doenhoff & Stivers 1945,
  NACA 0012 section), corrected for the closed trailing edge.
"""
import numpy as np
import pytest

from oracle import grid as G
from oracle import hermite as hm
from oracle import lattices as L
from oracle import solver as S
from paper_2504_04465_b300 import inputs as I


# ----------------------------------------------------------------------------- shock sensor
@pytest.mark.parametrize("tau", [0.5, 0.73])
def test_sensor_threshold_table(tau):
    """tau_eff = tau * alpha(eps): 1 below 0.01, 1.05 on [0.01, 0.1), A on [0.1, 1), 1/tau from 1."""
    A = 1.5
    eps = np.array([0.0, 0.009, 0.01, 0.0999, 0.1, 0.999, 1.0, 5.0])
    expect = np.array([tau, tau, 1.05 * tau, 1.05 * tau, A * tau, A * tau, 1.0, 1.0])
    got = tau * S.sensor_alpha(eps, tau, A)
    assert np.allclose(got, expect, rtol=0, atol=1e-15)
    # per-cell relaxation times broadcast with eps
    taus = np.full(eps.shape, tau)
    assert np.allclose(taus * S.sensor_alpha(eps, taus, 1.35),
                       np.where(eps >= 1, 1.0, taus * np.select([eps < 0.01, eps < 0.1, eps < 1], [1, 1.05, 1.35])),
                       rtol=0, atol=1e-15)


def test_sensor_eps_hand_values():
    """eps = (1/V) sum |f - f_eq| / f_eq over the V velocities of each cell."""
    # three velocities, two cells; cell 0: (0.1 + 0.5 + 1.0) / 3, cell 1: (0 + 0.25 + 0.5) / 3
    f = np.array([[1.1, 2.0], [0.5, 1.5], [2.0, 0.75]])
    feq = np.array([[1.0, 2.0], [1.0, 2.0], [1.0, 0.5]])
    assert np.allclose(S.sensor_eps(f, feq), [1.6 / 3, 0.75 / 3], rtol=0, atol=1e-15)


def test_sensor_eps_skips_vanishing_equilibria():
    """Terms whose f_eq is at or below 1e-300 contribute nothing; V still counts them (R10)."""
    f = np.array([[1.0], [3.0], [0.2]])
    feq = np.array([[0.0], [2.0], [1e-301]])
    assert S.sensor_eps(f, feq)[0] == pytest.approx(0.5 / 3, abs=1e-15)


# ----------------------------------------------------------------------------- boundary pass
def _bc_solver(latname, model, ext, faces, T0=None):
    lat = L.LATTICES[latname]
    spec = I.GridSpec(2, ext, 1, [], (False, False), faces)
    g = G.build(spec, lat)
    s = S.Solver(g, model, nu0=0.01, T0=T0)
    lv = g.levels[0]
    rng = np.random.default_rng(12)
    s.f[0] = rng.uniform(0.01, 0.2, (lat.Q, lv.n))
    if s.comp:
        s.g_[0] = rng.uniform(0.01, 0.2, (lat.Q, lv.n))
    return s, lv


def _at(lv, x, y):
    return int(lv.index[x, y])


def test_boundary_pass_d2q9_hand_set():
    """8x6 D2Q9 box: x- Dirichlet with extrapolated rho, x+ and y- Neumann, y+ Dirichlet."""
    faces = {"x-": ("dirichlet_rho", 1.3, (0.05, 0.01, 0.0)), "x+": ("neumann",),
             "y-": ("neumann",), "y+": ("dirichlet", 0.9, (0.02, -0.03, 0.0))}
    s, lv = _bc_solver("D2Q9", "rr", (8, 6), faces)
    lat = s.lat
    f0 = s.f[0].copy()
    s._boundaries(0)
    f1 = s.f[0]

    def eq(rho, u):
        return hm.feq_athermal(lat, np.array([rho]), np.array(u, float).reshape(2, 1))[:, 0]

    u_w, u_n = (0.05, 0.01), (0.02, -0.03)
    expect = {}
    # the interior (x 1..6, y 1..4) is untouched
    for x in range(1, 7):
        for y in range(1, 5):
            expect[(x, y)] = f0[:, _at(lv, x, y)]
    # x- layer, corners included: rho from the interior neighbour clamped into the interior
    for y in range(6):
        p = _at(lv, 1, min(max(y, 1), 4))
        expect[(0, y)] = eq(f0[:, p].sum(), u_w)
    # x+ layer (Neumann) except the top corner, which the Dirichlet face y+ takes
    for y in range(5):
        expect[(7, y)] = f0[:, _at(lv, 6, min(max(y, 1), 4))]
    # y- layer (Neumann) between the x faces
    for x in range(1, 7):
        expect[(x, 0)] = f0[:, _at(lv, x, 1)]
    # y+ layer (Dirichlet, imposed rho) including the corner shared with the Neumann face x+
    for x in range(1, 8):
        expect[(x, 5)] = eq(0.9, u_n)
    assert len(expect) == 48
    for (x, y), e in expect.items():
        assert np.allclose(f1[:, _at(lv, x, y)], e, rtol=0, atol=1e-15), (x, y)
    # the Dirichlet cells carry exactly the face's density and velocity
    c = _at(lv, 3, 5)
    assert f1[:, c].sum() == pytest.approx(0.9, abs=1e-15)
    assert np.allclose(lat.xi.T @ f1[:, c] / f1[:, c].sum(), u_n, atol=1e-15)
    c, p = _at(lv, 0, 2), _at(lv, 1, 2)
    assert f1[:, c].sum() == pytest.approx(f0[:, p].sum(), abs=1e-15)


def test_boundary_pass_d2q37_reach3_ddf():
    """10x8 D2Q37 box (reach 3): three boundary layers per face, f and g, default T = T0."""
    faces = {"x-": ("dirichlet", 1.2, (0.3, 0.05, 0.0), 0.8), "x+": ("neumann",),
             "y-": ("dirichlet_rho", 0.0, (0.1, 0.0, 0.0)), "y+": ("neumann",)}
    s, lv = _bc_solver("D2Q37", "poly_ddf", (10, 8), faces, T0=0.7)
    lat = s.lat
    f0, g0 = s.f[0].copy(), s.g_[0].copy()
    s._boundaries(0)
    cg = 2.0 / (1.4 - 1.0) - 2.0

    def eq(rho, u, T):
        return hm.feq_thermal(lat, np.array([rho]), np.array(u, float).reshape(2, 1), np.array([T]), 4)[:, 0]

    def clamp(x, y):
        return _at(lv, min(max(x, 3), 6), min(max(y, 3), 4))

    n_dir = n_neu = 0
    for x in range(10):
        for y in range(8):
            c = _at(lv, x, y)
            inner = 3 <= x <= 6 and 3 <= y <= 4
            if inner:
                assert np.array_equal(s.f[0][:, c], f0[:, c])
                continue
            if x <= 2:                     # x- Dirichlet wins every corner it touches
                ef = eq(1.2, (0.3, 0.05), 0.8)
                eg = cg * 0.8 * ef
                n_dir += 1
            elif y <= 2:                   # y- Dirichlet (rho extrapolated, T = T0)
                ef = eq(f0[:, clamp(x, y)].sum(), (0.1, 0.0), 0.7)
                eg = cg * 0.7 * ef
                n_dir += 1
            else:                          # x+ / y+ Neumann: copy the clamped interior cell
                ef, eg = f0[:, clamp(x, y)], g0[:, clamp(x, y)]
                n_neu += 1
            assert np.allclose(s.f[0][:, c], ef, rtol=0, atol=1e-15), (x, y)
            assert np.allclose(s.g_[0][:, c], eg, rtol=0, atol=1e-15), (x, y)
    assert n_dir == 3 * 8 + 7 * 3 and n_neu == 80 - 8 - n_dir


def test_uniform_inflow_channel_stays_uniform():
    """x- equilibrium inlet at the initial state, x+ Neumann: the uniform flow is a fixed point."""
    u = (0.05, 0.0, 0.0)
    faces = {"x-": ("dirichlet", 1.0, u), "x+": ("neumann",)}
    for extrap in (False, True):
        if extrap:
            faces["x-"] = ("dirichlet_rho", 7.0, u)     # the 7.0 must be ignored
        g = G.build(I.GridSpec(2, (24, 8), 1, [], (False, True), faces), L.D2Q9)
        s = S.Solver(g, "rr", nu0=0.02)
        n = g.levels[0].n
        s.init_fields([(np.ones(n), np.tile(np.array(u[:2])[:, None], (1, n)), None)])
        e = s.f[0][:, :1].copy()
        s.step_fine(30)
        assert np.abs(s.f[0] - e).max() < 1e-15


# ----------------------------------------------------------------------------- NACA 0012
# NACA Report 824, ordinates of the NACA 0012 section: x/c and y_t/c in per cent of the chord
NACA0012_X = [1.25, 2.5, 5.0, 7.5, 10, 15, 20, 25, 30, 40, 50, 60, 70, 80, 90, 95]
NACA0012_Y = [1.894, 2.615, 3.555, 4.200, 4.683, 5.345, 5.737, 5.941, 6.002, 5.803, 5.294, 4.563,
              3.664, 2.623, 1.448, 0.807]


def _column_half_thickness(xs, chord):
    """Half the number of solid cells in a one-cell-wide column at x/c = xs, in chords."""
    H = 2 * int(0.07 * chord) + 2
    spec = I.GridSpec(2, (1, H), 1, [], (True, True),
                      solids=[{"kind": "naca", "chord": float(chord), "x0": 0.5 - xs * chord,
                               "y0": H / 2, "t": 0.12}])
    m = G.solid_mask_level0(spec, (1, H))[0]
    n = int(m.sum())
    assert n % 2 == 0 and np.array_equal(m, m[::-1])        # symmetric about the chord
    return n / 2 / chord


def test_naca0012_ordinates():
    """Mask half-thickness = published ordinate to the table's rounding (0.5e-5 c) plus one cell.

    The published table is for the open trailing edge (x^4 coefficient -0.1015); reading R20
    closes the edge (-0.1036), which lowers y_t by 5 t (0.1036 - 0.1015) x^4 = 0.00126 x^4."""
    chord = 1_000_000
    for xp, yp in zip(NACA0012_X, NACA0012_Y):
        xs = xp / 100
        got = _column_half_thickness(xs, chord)
        closed = yp / 100 - 0.00126 * xs ** 4
        assert abs(got - closed) <= 0.55e-5 + 1.0 / chord, (xp, got, closed)


def test_naca0012_closed_edge_and_extent():
    chord = 10_000
    assert _column_half_thickness(-0.001, chord) == 0           # ahead of the leading edge
    assert _column_half_thickness(1.0005, chord) == 0           # behind the trailing edge
    assert _column_half_thickness(0.9999, chord) < 2.0 / chord  # closed trailing edge
    # maximum thickness 12 % of the chord at 30 % chord
    t = [_column_half_thickness(x / 100, chord) for x in range(20, 41)]
    assert 28 <= 20 + int(np.argmax(t)) <= 31
    assert abs(2 * max(t) - 0.12) < 2e-4
