"""Flow past a NACA0012 on three levels against the FP64 oracle (GPU required): the reduced forms
of the airfoil workloads (Sec. 6.3, transonic NACA0012 with the D2Q37 polynomial DDF; Sec. 6.4,
supersonic NACA0012 with the D2Q21 numerical equilibrium).

Chord 64 finest cells in a [-3C, 3C]^2 domain, the finest box [-0.25C, 1.25C] x [-0.3C, 0.3C],
the next [-0.75C, 2C] x [-0.75C, 0.75C].  These grids exercise what no periodic or tube case
does: the reach-3 staircase bounce-back of both 37- and 21-velocity lattices (links blocked by
any solid cell on their lattice segment, reading R11), equilibrium inlets and Neumann faces with
three boundary layers, refinement interfaces around a solid, and (D2Q21) the multipliers
coalesced and exploded next to the wall.  FP64 populations agree to 1e-12 (rounding order
only), element by element and within twice the reach of every interface and of the airfoil.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np
import pytest

from oracle import lattices as L
from paper_2504_04465_b300 import inputs as I
from tests import harness as H

pytestmark = pytest.mark.gpu

CHORD = 64
GAMMA = 1.4


def _spec(mach, T0, supersonic):
    return I.naca_spec(CHORD, mach, T0, GAMMA, n_levels=3, supersonic=supersonic, half_domain=3.0,
                       level_boxes=I.NACA_BOXES_SMALL)


def _fields(mach, T0):
    def fn(level, coords, c):
        return I.naca_fields(level, coords, mach, T0, GAMMA)
    return fn


# D2Q21, numerical equilibrium, Mach 1.5 supersonic inlet, T0 = 0.65 (the viscous reference
# temperature of the D2Q21 airfoil runs), Re 1e4 on the chord, sensor A = 1.35
M21, T21 = 1.5, 0.65
NU21 = M21 * np.sqrt(GAMMA * T21) * CHORD / 1e4
# D2Q37, polynomial equilibrium about c_s^2, Mach 0.8 subsonic inlet (density extrapolated)
M37, T37 = 0.8, L.D2Q37.cs2
NU37 = M37 * np.sqrt(GAMMA * T37) * CHORD / 1e4
N_FINE = 24          # six coarse steps of the three-level grid


@lru_cache(maxsize=None)
def oracle21(guess):
    return H.run_oracle(_spec(M21, T21, True), "D2Q21", "num_ddf", _fields(M21, T21), N_FINE, nu0=NU21, T0=T21,
                        gamma=GAMMA, sensor_A=1.35, guess=guess)


@lru_cache(maxsize=None)
def oracle37(sensor=True):
    return H.run_oracle(_spec(M37, T37, False), "D2Q37", "poly_ddf", _fields(M37, T37), N_FINE, nu0=NU37,
                        gamma=GAMMA, sensor_A=1.35 if sensor else None)


def _check_f64(sol, ctx, lam=False):
    err = H.compare_moments(sol, ctx)
    near = H.compare_near(sol, ctx)
    print("naca", sol.lat.Q, err, near)
    assert err["rho"] < 1e-12 and err["u"] < 1e-12 and err["T"] < 1e-12, err
    assert near["n"] > 0 and max(near["rho"], near["u"], near["T"]) < 1e-12, near
    tol = H.POP_TOL_NEWTON if sol.model == "num_ddf" else 1e-12
    assert H.compare_populations(sol, ctx, "f") < tol
    assert H.compare_populations(sol, ctx, "g") < tol


@pytest.mark.parametrize("guess", ["warm", "poly"])
def test_naca_d2q21_numerical_supersonic_f64(guess):
    sol = oracle21(guess)
    assert (sol.g.levels[0].ctype == 5).sum() > 300          # the airfoil is resolved
    assert sol.nonconv == 0
    ctx = H.make_gpu(_spec(M21, T21, True), "D2Q21", "num_ddf", "f64", _fields(M21, T21), nu0=NU21, T0=T21,
                     gamma=GAMMA, sensor_A=1.35, guess=guess)
    ctx.step_fine(N_FINE)
    ctx.sync()
    _check_f64(sol, ctx)
    s = ctx.stats()
    assert s.newton_nonconverged == 0 and s.newton_updates > 0
    ctx.close()


def test_naca_d2q37_polynomial_transonic_f64():
    sol = oracle37()
    ctx = H.make_gpu(_spec(M37, T37, False), "D2Q37", "poly_ddf", "f64", _fields(M37, T37), nu0=NU37,
                     gamma=GAMMA, sensor_A=1.35)
    ctx.step_fine(N_FINE)
    ctx.sync()
    _check_f64(sol, ctx)
    ctx.close()


@pytest.mark.parametrize("sensor", [False, True])
def test_naca_d2q37_polynomial_transonic_f32(sensor):
    """FP32 populations.  Sensor off: 1e-5 relative L2 and 3e-5 pointwise within twice the reach
    of the interfaces and the wall, the bounds of the other FP32 configurations.  Sensor on: the
    threshold flips of alpha(eps) (Eq. shock_function) that a rounding-sized difference can cause
    (tests/test_oracle_sensitivity.py); measured rho 8.9e-5, u 1.6e-4, T 4.9e-5 after 24 fine
    iterations, bound 5e-4."""
    sol = oracle37(sensor)
    ctx = H.make_gpu(_spec(M37, T37, False), "D2Q37", "poly_ddf", "f32", _fields(M37, T37), nu0=NU37,
                     gamma=GAMMA, sensor_A=1.35 if sensor else None)
    ctx.step_fine(N_FINE)
    ctx.sync()
    err = H.compare_moments(sol, ctx)
    near = H.compare_near(sol, ctx)
    print("naca d2q37 f32 sensor" if sensor else "naca d2q37 f32", err, near)
    l2, band = (5e-4, 5e-3) if sensor else (1e-5, 3e-5)
    assert err["rho"] < l2 and err["u"] < l2 and err["T"] < l2, err
    assert max(near["rho"], near["u"], near["T"]) < band, near
    ctx.close()
