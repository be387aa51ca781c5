"""FP32 populations against the FP64 oracle over 1000 fine iterations, for every lattice and
collision model of the path (GPU required).

Each case steps the oracle and the CUDA path side by side and compares them at 100, 250, 500
and 1000 fine iterations: the whole-domain relative L2 of rho, u and T, and the largest
pointwise error over the cells within twice the lattice reach of a refinement interface or a
solid, relative to the field's largest magnitude over the grid (``harness.compare_near``).
The curve is printed; the bounds asserted at 1000 iterations are the stated FP32 bounds of each
configuration.

Without the kinetic shock sensor every configuration meets 1e-5 at 1000 iterations, relative L2
and interface-local.  With the sensor on, the bound is the method's own sensitivity, not an
FP32 defect: alpha(eps) of Eq. shock_function jumps (1 to 1.05 at eps = 0.01, to A at 0.1, to
1/tau at 1), so a rounding-sized difference in a cell whose eps sits at a threshold changes its
relaxation time by 5 % or more, and the difference then spreads.  The FP64 oracle shows the same
growth when its populations get FP32-sized relative noise (2^-24) after every iteration
(tests/test_oracle_sensitivity.py); the bounds below are about twice the larger of that and the
measured FP32 gap.  When the first flip happens is a matter of chance: in |f - f_eq| / f_eq the
FP32 cancellation alone moves eps by about 1e-5 relative, so the onset differs from run to run
and between builds (the inviscid Sod tube has shown it before 100 and after 250 iterations).
"""
from __future__ import annotations

import pytest

from oracle import lattices as L
from tests import harness as H
from tests.test_gpu_d2q21_weak import NU0, W21_SPEC, weak_fields
from tests.test_gpu_d2q37_numerical import N37_SPEC, T0_VISC
from tests.test_gpu_parity import D3_SPEC, N21_SPEC, SOD_SPEC, TG_SPEC, d3_fields

pytestmark = pytest.mark.gpu

CHECKPOINTS = (100, 250, 500, 1000)


def _run(name, *args, **kw):
    sol, ctx, curve = H.error_curve(*args, CHECKPOINTS, **kw)
    for t, e in curve:
        print(name, t, {k: (f"{v:.2e}" if isinstance(v, float) else v) for k, v in e.items()})
    return sol, ctx, curve[-1][1]


def _check(err, bounds):
    assert err["near_n"] > 0
    for k, b in bounds.items():
        assert err[k] < b, (k, err[k], b, err)


@pytest.mark.parametrize("model", ["bgk", "rr"])
def test_d2q9_taylor_green_f32(model):
    _, ctx, err = _run("d2q9-" + model, TG_SPEC, "D2Q9", model, "f32", H.tg_fields(64, 2, seed=7, amp=0.01),
                       nu0=0.02)
    _check(err, {"rho": 1e-5, "u": 1e-5, "near_rho": 1e-5, "near_u": 1e-5})
    ctx.close()


def test_d3q27_sphere_f32():
    _, ctx, err = _run("d3q27", D3_SPEC, "D3Q27", "rr", "f32", d3_fields, nu0=0.01)
    _check(err, {"rho": 1e-5, "u": 1e-5, "near_rho": 1e-5, "near_u": 1e-5})
    ctx.close()


@pytest.mark.parametrize("model", ["bgk", "rr"])
def test_d2q13_weak_f32(model):
    _, ctx, err = _run("d2q13w-" + model, W21_SPEC, "D2Q13", model, "f32", weak_fields, nu0=NU0)
    _check(err, {"rho": 1e-5, "u": 1e-5, "near_rho": 1e-5, "near_u": 1e-5})
    ctx.close()


def test_d2q13_numerical_f32_populations():
    """Sensor off, T0 = 0.35."""
    _, ctx, err = _run("d2q13n", N21_SPEC, "D2Q13", "num_ddf", "f32", H.smooth_comp_fields((96, 64), 0.35),
                       nu0=0.01, T0=0.35)
    _check(err, {"rho": 1e-5, "u": 1e-5, "T": 1e-5, "near_rho": 3e-5, "near_u": 3e-5, "near_T": 3e-5})
    ctx.close()


@pytest.mark.parametrize("model", ["bgk", "rr"])
def test_d2q21_weak_f32(model):
    _, ctx, err = _run("d2q21w-" + model, W21_SPEC, "D2Q21", model, "f32", weak_fields, nu0=NU0)
    _check(err, {"rho": 1e-5, "u": 1e-5, "near_rho": 1e-5, "near_u": 1e-5})
    ctx.close()


# relative L2 1e-5; the largest pointwise error over the interface band (about 900 cells here)
# of an unbiased rounding noise runs 2 to 3 times its L2 norm in every configuration (D2Q9 and
# D3Q27 included), so the band maximum of the DDF models is held to 3e-5
TARGET = {"rho": 1e-5, "u": 1e-5, "T": 1e-5, "near_rho": 3e-5, "near_u": 3e-5, "near_T": 3e-5}


def test_d2q37_poly_smooth_f32():
    """D2Q37 thermal polynomial equilibrium, viscous, sensor off."""
    _, ctx, err = _run("d2q37-smooth", N37_SPEC, "D2Q37", "poly_ddf", "f32", H.smooth_comp_fields((96, 64), L.D2Q37.cs2),
                       nu0=0.01)
    _check(err, TARGET)
    ctx.close()


def test_d2q37_poly_sod_band_f32():
    """Inviscid Sod tube with the sensor: at 1000 iterations the measured gap was rho 2.4e-2 to
    3.3e-2, u 7.2e-3, T 2.1e-2 to 3.1e-2 over two builds (FP64 oracle with FP32-sized noise: 2.4e-2,
    6.0e-3, 2.4e-2)."""
    _, ctx, err = _run("d2q37-sod", SOD_SPEC, "D2Q37", "poly_ddf", "f32", H.sod_fields(256, L.D2Q37.cs2),
                       nu0=0.0, sensor_A=1.5)
    _check(err, {"rho": 8e-2, "u": 2e-2, "T": 8e-2, "near_rho": 1e-1, "near_u": 4e-2, "near_T": 8e-2})
    ctx.close()


@pytest.mark.parametrize("sensor", [False, True])
def test_d2q21_numerical_f32_populations(sensor):
    """Sensor off: 1e-5.  Sensor on (A = 1.35): measured rho 4.0e-5, u 4.9e-4, T 2.6e-5 at 1000
    iterations (noisy FP64 oracle: 4.1e-5, 5.0e-4, 2.5e-5)."""
    kw = {"sensor_A": 1.35} if sensor else {}
    _, ctx, err = _run("d2q21n-sensor" if sensor else "d2q21n", N21_SPEC, "D2Q21", "num_ddf", "f32",
                       H.smooth_comp_fields((96, 64), 0.9), nu0=0.01, T0=0.9, **kw)
    _check(err, {"rho": 1e-4, "u": 1.5e-3, "T": 1e-4, "near_rho": 4e-4, "near_u": 4e-3, "near_T": 3e-4} if sensor
           else TARGET)
    ctx.close()


@pytest.mark.parametrize("sensor", [False, True])
def test_d2q37_numerical_f32_populations(sensor):
    """Sensor off: 1e-5.  Sensor on (A = 1.35): measured u 9.2e-6 relative L2 and 4.8e-5 near the
    interface at 1000 iterations (noisy FP64 oracle: 6.4e-6 relative L2)."""
    kw = {"sensor_A": 1.35} if sensor else {}
    _, ctx, err = _run("d2q37n-sensor" if sensor else "d2q37n", N37_SPEC, "D2Q37", "num_ddf", "f32",
                       H.smooth_comp_fields((96, 64), T0_VISC), nu0=0.01, T0=T0_VISC, **kw)
    _check(err, {"rho": 1e-5, "u": 3e-5, "T": 1e-5, "near_rho": 2e-5, "near_u": 1.5e-4, "near_T": 1e-5} if sensor
           else TARGET)
    ctx.close()
