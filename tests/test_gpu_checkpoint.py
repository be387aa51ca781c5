"""Checkpoint/restart and variant tuning through the C ABI: a run restored from a checkpoint
continues bitwise like the run that wrote it; a checkpoint of another configuration is refused."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2504_04465_b300 import inputs as I
from tests import harness as H

pytestmark = pytest.mark.gpu

SPEC = I.GridSpec(2, (256, 256), 3, [(1, (64, 64), (192, 192)), (0, (96, 96), (160, 160))], (True, True))


def fields(level, coords, c):
    return I.taylor_green_fields(c, 64, 3, 0.05, 1.0 / 3.0)


@pytest.mark.parametrize("storage", ["f32", "f16dev", "f64"])
def test_restart_continues_bitwise(storage, tmp_path):
    path = str(tmp_path / "state.ckpt")
    a = H.make_gpu(SPEC, "D2Q9", "rr", storage, fields, nu0=0.08)
    a.step_fine(7)                     # not at a coarse synchronisation instant
    a.save(path)
    a.step_fine(9)
    a.sync()
    b = H.make_gpu(SPEC, "D2Q9", "rr", storage, lambda lv, co, c: (np.ones(co.shape[0]), np.zeros((2, co.shape[0]))),
                   nu0=0.08)
    b.load(path)
    b.step_fine(9)
    b.sync()
    assert np.array_equal(a.populations("f"), b.populations("f"))
    assert a.stats().fine_iterations == b.stats().fine_iterations == 16


def test_checkpoint_of_another_configuration_is_refused(tmp_path):
    from paper_2504_04465_b300.lbmtree import LbmError
    path = str(tmp_path / "state.ckpt")
    a = H.make_gpu(SPEC, "D2Q9", "rr", "f32", fields, nu0=0.08)
    a.save(path)
    b = H.make_gpu(SPEC, "D2Q9", "rr", "f64", fields, nu0=0.08)
    with pytest.raises(LbmError):
        b.load(path)


def test_autotune_selects_a_compiled_variant():
    ctx = H.make_gpu(SPEC, "D2Q9", "rr", "f32", fields, nu0=0.08)
    best, ms = ctx.autotune(2)
    assert 0 <= best < len(ctx.variants())
    assert len(ms) == len(ctx.variants()) and all(m > 0 for m in ms)
    assert ms[best] == min(ms)


def test_grid_arrays_from_the_torch_caching_allocator():
    import torch
    from paper_2504_04465_b300 import lbmtree as lt
    a = H.make_gpu(SPEC, "D2Q9", "rr", "f32", fields, nu0=0.08)
    before = torch.cuda.memory_allocated(0)
    ctx = lt.Context(2, device=0)
    alloc = lt.torch_allocator(0)
    ctx.set_allocator(alloc)
    ctx.configure(SPEC, "D2Q9", "rr", "f32", nu0=0.08)
    assert torch.cuda.memory_allocated(0) - before >= ctx.stats().device_bytes > 0
    lv, xyz, ty = ctx.cells()
    rho = np.ones(lv.size)
    u = np.zeros((2, lv.size))
    for level in np.unique(lv):
        m = lv == level
        r, uu = fields(int(level), xyz[m, :2], I.cell_centres(xyz[m, :2], int(level)))
        rho[m], u[:, m] = r, uu
    ctx.init_fields(rho, u)
    a.step_fine(12)
    ctx.step_fine(12)
    a.sync()
    ctx.sync()
    assert np.array_equal(a.populations("f"), ctx.populations("f"))
    ctx.close()
