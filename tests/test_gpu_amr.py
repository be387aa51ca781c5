"""Adaptive mesh refinement against the oracle (GPU required): grids built from level maps
(Sec. 8's mesh density field; disc-shaped regions with staircase borders), the kinetic-sensor
criterion, and remeshing a running state by copy, uniform explosion and coalescence.

FP64: the state right after a remesh and after further steps matches the oracle's remesh to
1e-12 (populations element-wise, the Newton-solved ones to ten times the Newton tolerance); the
ledger is the same before and after a remesh to 1e-13; the sensor maps are identical."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import amr
from oracle import lattices as L
from paper_2504_04465_b300 import inputs as I
from tests import harness as H

pytestmark = pytest.mark.gpu


def disc_map(n, centre, radius, levels, lat):
    x, y = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    r = np.hypot(x - centre[0], y - centre[1])
    raw = np.where(r < radius, 0, levels - 1).astype(np.uint8)
    return amr.grade(raw, levels, L.LATTICES[lat].reach, (True, True))


def vortex_fields(n, T0=None):
    def fn(level, coords, c):
        x, y = c[:, 0] - 0.4 * n, c[:, 1] - 0.5 * n
        r2 = (x * x + y * y) / (0.08 * n) ** 2
        g = 0.05 * np.exp(-0.5 * r2)
        rho = 1.0 - 0.5 * g * g
        u = np.stack([0.05 - g * y / (0.08 * n), g * x / (0.08 * n)])
        if T0 is None:
            return rho, u
        return rho, u, np.full(rho.size, T0)
    return fn


CASES = [
    ("D2Q9", "rr", 3, {}, None),
    ("D2Q21", "num_ddf", 2, {"T0": 0.9, "sensor_A": 1.35}, 0.9),
    ("D2Q37", "poly_ddf", 3, {}, "cs2"),
]


def _spec(n, m, levels):
    return I.GridSpec(2, (n, n), levels, [], (True, True), level_map=m)


@pytest.mark.parametrize("lat,model,levels,kw,T0", CASES, ids=[c[0] for c in CASES])
def test_remesh_matches_oracle(lat, model, levels, kw, T0):
    n = 128
    if T0 == "cs2":
        T0 = L.LATTICES[lat].cs2
    fields = vortex_fields(n, T0)
    nu = 0.01
    m1 = disc_map(n, (0.4 * n, 0.5 * n), 14, levels, lat)
    m2 = disc_map(n, (0.5 * n, 0.55 * n), 14, levels, lat)
    P = 2 ** (levels - 1)
    sol = H.run_oracle(_spec(n, m1, levels), lat, model, fields, 2 * P, nu0=nu, **kw)
    ctx = H.make_gpu(_spec(n, m1, levels), lat, model, "f64", fields, nu0=nu, **kw)
    ctx.step_fine(2 * P)
    ctx.sync()
    led0 = ctx.conserved()
    sol2 = amr.remesh(sol, _spec(n, m2, levels))
    ctx.remesh(m2)
    led1 = ctx.conserved()
    tol = H.POP_TOL_NEWTON if model == "num_ddf" else 1e-12
    assert H.compare_populations(sol2, ctx, "f") < tol
    if model != "rr":
        assert H.compare_populations(sol2, ctx, "g") < tol
    k = 3 if model == "rr" else 4
    assert np.abs(led1[:k] - led0[:k]).max() <= 1e-13 * led0[0] * (1 if model != "num_ddf" else 100)
    sol2.step_fine(2 * P)
    ctx.step_fine(2 * P)
    ctx.sync()
    err = H.compare_moments(sol2, ctx)
    print("remesh", lat, model, err)
    assert err["rho"] < 1e-12 and err["u"] < 1e-12, err
    assert H.compare_populations(sol2, ctx, "f") < tol
    ctx.close()


def test_sensor_level_map_matches_oracle():
    """The GPU sensor map of a Sod state equals the oracle's (threshold 0.2)."""
    lat = "D2Q21"
    n = 128
    m0 = np.ones((n, 32), np.uint8)
    spec = I.GridSpec(2, (n, 32), 2, [], (True, True), level_map=m0)

    def fields(level, coords, c):
        rho, u, T = I.sod_fields(c, n, 0.9)
        far = c[:, 0] > 0.75 * n
        return np.where(far, 1.0, rho), u, np.where(far, 0.9, T)
    kw = dict(nu0=0.0, T0=0.9, sensor_A=1.5)
    sol = H.run_oracle(spec, lat, "num_ddf", fields, 8, **kw)
    ctx = H.make_gpu(spec, lat, "num_ddf", "f64", fields, **kw)
    ctx.step_fine(8)
    ctx.sync()
    mo = amr.sensor_level_map(sol, 0.2)
    mg = ctx.amr_level_map(0.2)
    assert (mo == 0).sum() > 0
    assert np.array_equal(mo, mg)
    ctx.close()


def test_vortex_follows_the_refinement():
    """The paper's convected-vortex check (Sec. 8), small: a refined disc follows a vortex carried
    by a uniform flow, remeshed every two coarse steps; the GPU run stays equal to the oracle's
    and the mass of the periodic box stays constant across the remeshes."""
    lat, model, levels, n = "D2Q9", "rr", 2, 128
    fields = vortex_fields(n)
    centre = np.array([0.4 * n, 0.5 * n])
    m = disc_map(n, centre, 16, levels, lat)
    sol = H.run_oracle(_spec(n, m, levels), lat, model, fields, 0, nu0=1e-4)
    ctx = H.make_gpu(_spec(n, m, levels), lat, model, "f64", fields, nu0=1e-4)
    mass0 = ctx.conserved()[0]
    for k in range(4):
        sol.step_coarse(2)
        ctx.step(2)
        centre = centre + np.array([0.05 * 2 * 2, 0.0])            # u_x = 0.05, 2 coarse steps of 2
        m = disc_map(n, centre, 16, levels, lat)
        sol = amr.remesh(sol, _spec(n, m, levels))
        ctx.remesh(m)
    sol.step_coarse(2)
    ctx.step(2)
    ctx.sync()
    err = H.compare_moments(sol, ctx)
    print("vortex amr", err)
    assert err["rho"] < 1e-12 and err["u"] < 1e-12, err
    assert abs(ctx.conserved()[0] - mass0) <= 1e-13 * mass0
    ctx.close()


def test_remesh_identity_at_size():
    """A 2048^2 D2Q9 RR state on a three-level disc map, remeshed onto the same map: bulk and
    boundary cells keep their moments bit for bit and the totals are unchanged (a property at
    any size)."""
    lat, n, levels = "D2Q9", 2048, 3
    m = disc_map(n, (0.5 * n, 0.5 * n), 200, levels, lat)
    spec = _spec(n, m, levels)
    ctx = H.make_gpu(spec, lat, "rr", "f64", vortex_fields(n), nu0=0.01)
    ctx.step(4)
    ctx.sync()
    r0 = ctx.moments()
    t0 = ctx.conserved()
    _, _, ty = ctx.cells()
    ctx.remesh(m)
    r1 = ctx.moments()
    keep = np.isin(ty, (1, 4))
    assert np.array_equal(r0[0][keep], r1[0][keep]) and np.array_equal(r0[1][:, keep], r1[1][:, keep])
    assert np.abs(ctx.conserved()[:3] - t0[:3]).max() <= 1e-13 * t0[0]
    ctx.close()
