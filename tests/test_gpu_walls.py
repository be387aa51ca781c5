"""Wall faces against the FP64 oracle (GPU required): halfway bounce-back at the face planes
with Ladd's moving-wall term (Appendix A.3; the lid-driven cavity of Sec. 5.1), on uniform and
two-level D2Q9, D2Q13 and D3Q27 cavities, a plane Couette channel and a closed D2Q37 box
(reach-3 bounce-back of both distributions).

FP64 moments and populations agree to 1e-12 and the cavity's mass stays constant to 1e-13 while
the lid drives it; FP32 deviations stay below 1e-5."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2504_04465_b300 import inputs as I
from tests import harness as H

pytestmark = pytest.mark.gpu


def rest(level, coords, c):
    return np.ones(c.shape[0]), np.zeros((c.shape[1], c.shape[0]))


CASES = [
    ("cavity_q9_two_level_rr", I.cavity_spec(64, 0.1, 2, (16, 48)), "D2Q9", "rr", 40, {}),
    ("cavity_q9_trt", I.cavity_spec(32, 0.1), "D2Q9", "trt", 40, {}),
    ("cavity_q13_bgk", I.cavity_spec(32, 0.1), "D2Q13", "bgk", 40, {}),
    ("cavity_q27_two_level_rr", I.cavity_spec(32, 0.05, 2, (8, 24), dim=3), "D3Q27", "rr", 12, {}),
    ("couette_q9_bgk", I.couette_spec(16, 16, 0.05), "D2Q9", "bgk", 200, {}),
]


@pytest.mark.parametrize("name,spec,lat,model,n,kw", CASES, ids=[c[0] for c in CASES])
def test_walls_f64(name, spec, lat, model, n, kw):
    sol = H.run_oracle(spec, lat, model, rest, n, nu0=0.02, **kw)
    ctx = H.make_gpu(spec, lat, model, "f64", rest, nu0=0.02, **kw)
    m0 = ctx.conserved()[0]
    ctx.step_fine(n)
    ctx.sync()
    err = H.compare_moments(sol, ctx)
    near = H.compare_near(sol, ctx) if spec.n_levels > 1 else {"n": 1, "rho": 0.0, "u": 0.0}
    print(name, err, near)
    assert err["rho"] < 1e-12 and err["u"] < 1e-12, err
    assert near["n"] > 0 and near["rho"] < 1e-12 and near["u"] < 1e-12, near
    assert H.compare_populations(sol, ctx) < 1e-12
    assert abs(ctx.conserved()[0] - m0) <= 1e-13 * m0
    ctx.close()


def test_cavity_f32():
    spec = I.cavity_spec(64, 0.1, 2, (16, 48))
    sol = H.run_oracle(spec, "D2Q9", "rr", rest, 40, nu0=0.02)
    ctx = H.make_gpu(spec, "D2Q9", "rr", "f32", rest, nu0=0.02)
    ctx.step_fine(40)
    ctx.sync()
    err = H.compare_moments(sol, ctx)
    print("cavity f32", err)
    assert err["rho"] < 1e-5 and err["u"] < 1e-5, err
    ctx.close()


def test_closed_box_d2q37_f64():
    """A Sod tube closed by resting walls at both ends: reach-3 bounce-back of f and g, inviscid
    with the kinetic sensor (A = 1.5; without it the shock reflected at the wall drives the
    inviscid polynomial model unstable within 40 iterations, on the oracle as well)."""
    from paper_2504_04465_b300 import lbmtree as lt
    faces = {f: ("wall", 1.0, (0.0, 0.0, 0.0)) for f in ("x-", "x+")}
    spec = I.GridSpec(2, (128, 32), 1, [], (False, True), faces)
    T0 = lt.lattice_cs2("D2Q37")

    def fields(level, coords, c):
        return I.sod_fields(c, 128, T0)
    sol = H.run_oracle(spec, "D2Q37", "poly_ddf", fields, 40, nu0=0.0, sensor_A=1.5)
    ctx = H.make_gpu(spec, "D2Q37", "poly_ddf", "f64", fields, nu0=0.0, sensor_A=1.5)
    t0 = ctx.conserved()
    ctx.step_fine(40)
    ctx.sync()
    err = H.compare_moments(sol, ctx)
    print("closed box d2q37", err)
    assert err["rho"] < 1e-12 and err["u"] < 1e-12 and err["T"] < 1e-12, err
    assert H.compare_populations(sol, ctx, "f") < 1e-12
    assert H.compare_populations(sol, ctx, "g") < 1e-12
    t1 = ctx.conserved()
    assert abs(t1[0] - t0[0]) <= 1e-13 * t0[0]
    ctx.close()


def test_cavity_mass_at_size():
    """A 1024^2 lid-driven cavity with a centred refined patch (two levels, RR, FP64): the mass
    stays constant to round-off over 50 coarse steps while the lid drives the flow."""
    spec = I.cavity_spec(1024, 0.1, 2, (256, 768))
    ctx = H.make_gpu(spec, "D2Q9", "rr", "f64", rest, nu0=0.05)
    t0 = ctx.conserved()
    ctx.step(50)
    t1 = ctx.conserved()
    assert abs(t1[0] - t0[0]) <= 1e-12 * t0[0]
    assert abs(t1[1]) > 1e-3
    ctx.close()
