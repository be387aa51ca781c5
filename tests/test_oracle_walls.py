"""Pins of the oracle's wall faces (CPU only): halfway bounce-back at the face plane with Ladd's
moving-wall term (Appendix A.3, Sec. 5.1), checked against the exact plane Couette profile,
mass conservation in a lid-driven cavity (2D and 3D, uniform and refined) and a closed box of
the compressible double distribution."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import grid as G
from oracle import lattices as L
from oracle import solver as S
from paper_2504_04465_b300 import inputs as I


@pytest.mark.parametrize("model", ["bgk", "rr", "trt"])
def test_couette_profile_is_linear(model):
    """Halfway bounce-back puts the walls at the face planes y = 0 and y = ny; the steady plane
    Couette profile is then u_x = U y / ny at the cell centres, whatever tau."""
    nx, ny, U = 4, 8, 0.05
    lat = L.D2Q9
    g = G.build(I.couette_spec(nx, ny, U), lat)
    s = S.Solver(g, model, nu0=1.0 / 6.0)           # tau = 1
    lv = g.levels[0]
    s.init_fields([(np.ones(lv.n), np.zeros((2, lv.n)), None)])
    s.step_fine(4000)
    rho, u, _ = s.moments(0)
    y = lv.coords[:, 1] + 0.5
    assert np.abs(u[0] - U * y / ny).max() < 1e-9 * U
    assert np.abs(u[1]).max() < 1e-12


@pytest.mark.parametrize("spec,lat,model", [
    (I.cavity_spec(32, 0.1), L.D2Q9, "rr"),
    (I.cavity_spec(64, 0.1, 2, (16, 48)), L.D2Q9, "rr"),
    (I.cavity_spec(32, 0.1), L.D2Q13, "bgk"),
    (I.cavity_spec(16, 0.05, dim=3), L.D3Q27, "rr"),
])
def test_lid_driven_cavity_keeps_mass(spec, lat, model):
    """The wall terms of a link pair at a lid cell cancel, and the two lid corners (links
    leaving through the lid and a side wall take half the lid velocity, reading R38) cancel each
    other: the mass of the closed cavity is constant to round-off while the lid drives it."""
    g = G.build(spec, lat)
    s = S.Solver(g, model, nu0=0.02)
    s.init_fields([(np.ones(lv.n), np.zeros((lat.D, lv.n)), None) for lv in g.levels])
    m0 = s.ledger()
    s.step_coarse(20)
    m1 = s.ledger()
    assert abs(m1[0] - m0[0]) < 1e-13 * m0[0]
    assert abs(m1[1]) > 1e-4 * m0[0]          # the lid has put x momentum in


def test_wall_corner_links_take_the_mean_velocity():
    lat = L.D2Q9
    g = G.build(I.cavity_spec(8, 0.1), lat)
    lv = g.levels[0]
    k = lv.index[0, 7]                          # top-left fluid cell
    q = [j for j in range(lat.Q) if tuple(lat.xi[j]) == (1, -1)][0]    # source (-1, 8): lid and x-
    assert lv.blocked[q, k]
    assert abs(lv.wall_term[q, k] - 2 * lat.w[q] * 0.5 * 0.1 / lat.cs2) < 1e-15
    q2 = [j for j in range(lat.Q) if tuple(lat.xi[j]) == (-1, -1)][0]  # source (1, 8): lid only
    assert abs(lv.wall_term[q2, k] + 2 * lat.w[q2] * 0.1 / lat.cs2) < 1e-15


def test_closed_box_compressible():
    """Stationary walls around the D2Q37 double distribution (a Sod tube closed at both ends):
    mass is kept to round-off and energy to the round-off of the collisions."""
    lat = L.D2Q37
    faces = {f: ("wall", 1.0, (0.0, 0.0, 0.0)) for f in ("x-", "x+")}
    spec = I.GridSpec(2, (128, 8), 1, [], (False, True), faces)
    g = G.build(spec, lat)
    s = S.Solver(g, "poly_ddf", nu0=0.0, sensor_A=1.5)
    lv = g.levels[0]
    c = I.cell_centres(lv.coords, 0)
    rho, u, T = I.sod_fields(c, 128, lat.cs2)
    s.init_fields([(rho, u, T)])
    m0 = s.ledger()
    s.step_fine(40)
    m1 = s.ledger()
    assert abs(m1[0] - m0[0]) < 1e-13 * m0[0]
    # energy: each collision keeps it to the round-off of the 37-term equilibrium sums
    assert abs(m1[-1] - m0[-1]) < 1e-11 * abs(m0[-1])


def test_ghosts_near_a_wall_are_refused():
    with pytest.raises(G.GridError):
        G.build(I.cavity_spec(64, 0.1, 2, (0, 32)), L.D2Q9)
