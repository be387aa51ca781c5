"""Failure detection without a GPU fault: a Newton solve that cannot converge in its iteration
budget sets the device status word that lbm_sync reports; a NaN in the state makes the FP64
conservation totals non-finite, which lbm_conserved reports.  Both leave the context usable."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2504_04465_b300 import inputs as I
from tests import harness as H
from tests.test_gpu_parity import N21_SPEC

pytestmark = pytest.mark.gpu


def test_unconverged_newton_is_reported_and_the_context_stays_usable():
    from paper_2504_04465_b300.lbmtree import LbmError, ERR
    fn = H.smooth_comp_fields((96, 64), 0.9)
    ctx = H.make_gpu(N21_SPEC, "D2Q21", "num_ddf", "f64", fn, nu0=0.01, T0=0.9, guess="zero")
    ctx.set_newton_precision(False, 1e-300)      # a tolerance no FP64 residual reaches
    ctx.step_fine(1)
    with pytest.raises(LbmError) as e:
        ctx.sync()
    assert ERR[e.value.code] == "NEWTON"
    assert ctx.stats().newton_nonconverged > 0
    rho, u, T = ctx.moments()                    # results are still written
    assert np.isfinite(rho).all()


def test_nonfinite_state_is_reported_by_the_ledger():
    from paper_2504_04465_b300.lbmtree import LbmError, ERR

    def fields(level, coords, c):
        rho, u = I.taylor_green_fields(c, 32, 2, 0.05, 1.0 / 3.0)
        if level == 0:
            rho = rho.copy()
            rho[0] = np.nan
        return rho, u
    ctx = H.make_gpu(I.taylor_green_spec(32, 8, 24, 2), "D2Q9", "rr", "f64", fields, nu0=0.02)
    with pytest.raises(LbmError) as e:
        ctx.conserved()
    assert ERR[e.value.code] == "NONFINITE"
    ctx.step(1)                                  # still usable
    ctx.sync()
