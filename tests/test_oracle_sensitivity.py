"""How the FP64 oracle responds to rounding-sized perturbations, with and without the kinetic
shock sensor: the reason the FP32 parity bounds of the sensor configurations are wider than
1e-5 (tests/test_gpu_fp32_long.py).

alpha(eps) of Eq. shock_function is a step function of eps (1, 1.05, A, 1/tau on the bands
split at 0.01, 0.1 and 1), so the map from one iteration to the next is discontinuous: two runs
whose populations differ by rounding can relax a cell whose eps sits at a threshold with
relaxation times 5 % or more apart.  Here the FP64 oracle runs the D2Q21 numerical-equilibrium
case of the FP32 parity test twice, once with fresh relative noise of the FP32 unit roundoff
(2^-24) on every population after every fine iteration.  Without the sensor the two runs stay
within about 1e-6 of each other in u (measured 8e-7: the noise accumulates, the viscous
relaxation damps it); with it they part by about 4e-4, as the FP32 CUDA path parts from the FP64
oracle.
"""
import numpy as np
import pytest

from oracle import grid as G
from tests import harness as H
from tests.test_gpu_parity import N21_SPEC

N_FINE = 300


def _pair(sensor_A):
    fn = H.smooth_comp_fields((96, 64), 0.9)
    kw = dict(nu0=0.01, T0=0.9) if sensor_A is None else dict(nu0=0.01, T0=0.9, sensor_A=sensor_A)
    clean = H.run_oracle(N21_SPEC, "D2Q21", "num_ddf", fn, N_FINE, **kw)
    noisy = H.run_oracle(N21_SPEC, "D2Q21", "num_ddf", fn, 0, **kw)
    rng = np.random.default_rng(2 ** 24)
    for _ in range(N_FINE):
        noisy.step_fine(1)
        for lev in range(len(noisy.g.levels)):
            noisy.f[lev] *= 1 + 2.0 ** -24 * rng.uniform(-1, 1, noisy.f[lev].shape)
            noisy.g_[lev] *= 1 + 2.0 ** -24 * rng.uniform(-1, 1, noisy.g_[lev].shape)
    num = den = 0.0
    for lev, lv in enumerate(clean.g.levels):
        m = np.isin(lv.ctype, (G.FLUID, G.BC))
        a, b = clean.moments(lev)[1][:, m], noisy.moments(lev)[1][:, m]
        num += ((a - b) ** 2).sum()
        den += (a ** 2).sum()
    return (num / den) ** 0.5


@pytest.mark.slow
def test_sensor_amplifies_rounding_noise():
    off = _pair(None)
    on = _pair(1.35)
    print("relative L2 of u between the clean and the noisy run: sensor off %.2e, on %.2e" % (off, on))
    assert off < 3e-6
    assert on > 3e-5
