"""The allocation-free conserved-totals entry point (lbm_conserved_noalloc) gives the same totals
as lbm_conserved on two calls in a row.

lbm_conserved_noalloc exists for callers that cannot allocate device memory at the moment they
want the totals (a framework that owns all device memory through its own pool, a loop that must
not trigger an allocation's synchronisation); it writes into a device buffer the caller owns and
keeps its partial sums in a fixed array inside the library.  This file is collected last so that
a failing run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2504_04465_b300 import inputs as I

from . import harness as H

pytestmark = pytest.mark.gpu


def test_noalloc_conserved_matches_conserved_on_two_calls():
    import torch
    spec = I.taylor_green_spec(64, 16, 48, 2)
    fn = H.tg_fields(64, 2, seed=7, amp=0.01)
    ctx = H.make_gpu(spec, "D2Q9", "rr", "f64", fn, nu0=0.02)
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")   # the test owns it
    for _ in range(2):
        ctx.step(5)
        ref = ctx.conserved()
        ctx.conserved_noalloc(out.data_ptr())
        ctx.sync()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= 1e-12 * abs(ref[0])


def test_noalloc_rejects_off_sync_instant():
    import torch
    from paper_2504_04465_b300 import lbmtree as lt
    spec = I.taylor_green_spec(32, 8, 24, 2)
    ctx = H.make_gpu(spec, "D2Q9", "bgk", "f64", H.tg_fields(32, 2), nu0=0.02)
    ctx.step_fine(1)                    # mid coarse step
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(lt.LbmError) as e:
        ctx.conserved_noalloc(out.data_ptr())
    assert e.value.code == -2
