"""Batched stepping of several uneven cases (lbm_batch_*): bitwise equal to stepping each case
on its own, with and without the captured schedule graph, across groups of different lattices
and storage formats, and (through that) equal to the FP64 oracle on two of the cases."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2504_04465_b300 import inputs as I
from tests import harness as H

pytestmark = pytest.mark.gpu

SMALL = ["tg0", "sod1", "tg10", "sod11", "tg22", "sod25"]


def small_cases():
    by = {c["name"]: c for c in I.batch_cases()}
    return [by[k] for k in SMALL]


def make(case, storage, variant=0):
    ctx = H.make_gpu(case["spec"], case["lattice"], case["model"], storage, lambda lv, co, c: case["fields"](lv, co),
                     **case["params"])
    if variant:
        ctx.set_variant(variant)
    return ctx


def populations(ctx, comp):
    out = [ctx.populations("f")]
    if comp:
        out.append(ctx.populations("g"))
    return out


def assert_same(a, b, comp):
    for x, y in zip(populations(a, comp), populations(b, comp)):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("graph", [False, True])
def test_batch_equals_individual_steps_f64(graph):
    from paper_2504_04465_b300.lbmtree import Batch
    cases = small_cases()
    solo = [make(c, "f64") for c in cases]
    together = [make(c, "f64") for c in cases]
    b = Batch(together)
    b.use_graph(graph)
    info = b.info()
    assert info["groups"] == 2 and info["span"] == 16
    n = 2 * info["span"] + 3
    b.step_fine(n)
    b.sync()
    for s in solo:
        s.step_fine(n)
        s.sync()
    # two launches (interior + general) per group per fine iteration at most
    assert b.info()["launches"] <= 2 * 2 * n
    for c, s, t in zip(cases, solo, together):
        assert_same(s, t, c["model"] == "poly_ddf")
        assert t.stats().fine_iterations == n


def test_batch_matches_oracle_and_survives_solo_steps():
    from paper_2504_04465_b300.lbmtree import Batch
    cases = small_cases()
    ctxs = [make(c, "f64") for c in cases]
    b = Batch(ctxs)
    b.use_graph(True)
    b.step_fine(16)
    ctxs[2].step_fine(3)          # one case advances on its own in between
    b.step_fine(21)
    b.sync()
    for k, n in ((2, 40), (5, 37)):
        c = cases[k]
        sol = H.run_oracle(c["spec"], c["lattice"], c["model"], lambda lv, co, cc: c["fields"](lv, co), n,
                           **c["params"])
        err = H.compare_moments(sol, ctxs[k])
        assert all(v < 1e-12 for v in err.values()), (c["name"], err)


def test_batch_f32_with_variant_equals_individual():
    from paper_2504_04465_b300.lbmtree import Batch
    cases = [c for c in small_cases() if c["lattice"] == "D2Q9"]
    solo = [make(c, "f32", variant=2) for c in cases]
    together = [make(c, "f32", variant=2) for c in cases]
    b = Batch(together)
    b.use_graph(True)
    b.step_fine(40)
    b.sync()
    for s in solo:
        s.step_fine(40)
        s.sync()
    for s, t in zip(solo, together):
        assert_same(s, t, False)


@pytest.mark.parametrize("storage", ["f16dev", "f32"])
def test_batch_mixed_lattices_equal_individual(storage):
    """D2Q9 (binary16 storage value written by the collision) and D2Q37 groups in one batch."""
    from paper_2504_04465_b300.lbmtree import Batch
    cases = small_cases()
    solo = [make(c, storage) for c in cases]
    together = [make(c, storage) for c in cases]
    b = Batch(together)
    b.use_graph(True)
    b.step_fine(35)
    b.sync()
    for s in solo:
        s.step_fine(35)
        s.sync()
    for c, s, t in zip(cases, solo, together):
        assert_same(s, t, c["model"] == "poly_ddf")


def test_batch_rejects_lattices_without_batched_kernels():
    from paper_2504_04465_b300.lbmtree import Batch, LbmError
    spec = I.sphere_spec(4)
    ctx = H.make_gpu(spec, "D3Q27", "rr", "f32", lambda lv, co, c: I.sphere_fields(lv, co), nu0=I.sphere_nu0(4))
    with pytest.raises(LbmError):
        Batch([ctx])
