"""D2Q21 weakly compressible BGK and recursive regularization (Appendix A.2; the D2Q21 Hermite
basis is every tensor component up to order 3, c_s^2 = 2/3) against the FP64 oracle on a
two-level periodic grid.

Tolerances: FP64 populations agree to 1e-12 relative L2 (rounding order only) and conserve mass
and momentum across the refinement interface to round-off; FP32 deviations to 1e-5 for rho and u
over 20 fine iterations here and over 1000 in tests/test_gpu_fp32_long.py."""
from __future__ import annotations

from functools import lru_cache

import numpy as np
import pytest

from paper_2504_04465_b300 import inputs as I
from tests import harness as H

pytestmark = pytest.mark.gpu

W21_SPEC = I.GridSpec(2, (96, 64), 2, [(0, (32, 16), (64, 48))], (True, True))
NU0 = 0.02


def weak_fields(level, coords, c):
    """rho with a Gaussian bump, a uniform stream with a sinusoidal cross flow, 1e-2 seeded
    perturbation of u."""
    rho = 1 + 0.01 * np.exp(-((c - np.array([48.0, 32.0])) ** 2).sum(1) / 64)
    u = np.stack([0.05 + 0 * rho, 0.02 * np.sin(2 * np.pi * c[:, 0] / 96)])
    u = u + 1e-2 * np.stack([I.uniform_at(2121, level, coords, k) for k in range(2)])
    return rho, u


@lru_cache(maxsize=None)
def oracle(model):
    return H.run_oracle(W21_SPEC, "D2Q21", model, weak_fields, 20, nu0=NU0)


@pytest.mark.parametrize("model", ["rr", "bgk"])
def test_d2q21_weak_f64(model):
    sol = oracle(model)
    ctx = H.make_gpu(W21_SPEC, "D2Q21", model, "f64", weak_fields, nu0=NU0)
    t0 = ctx.conserved()
    ctx.step(10)
    err = H.compare_moments(sol, ctx)
    print("d2q21", model, "f64", err)
    assert err["rho"] < 1e-12 and err["u"] < 1e-12, err
    t1 = ctx.conserved()
    assert abs(t1[0] - t0[0]) <= 1e-13 * abs(t0[0])       # mass, exactly conserved (R1, R3)
    assert np.abs(t1[1:3] - t0[1:3]).max() <= 1e-13 * abs(t0[0])   # momentum across the interface
    ctx.close()


@pytest.mark.parametrize("model", ["rr", "bgk"])
def test_d2q21_weak_f32(model):
    sol = oracle(model)
    ctx = H.make_gpu(W21_SPEC, "D2Q21", model, "f32", weak_fields, nu0=NU0)
    ctx.step(10)
    err = H.compare_moments(sol, ctx)
    print("d2q21", model, "f32", err)
    assert err["rho"] < 1e-5 and err["u"] < 1e-5, err
    ctx.close()
