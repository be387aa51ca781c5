"""Pins of the oracle's adaptive mesh refinement (CPU only): the level-map regions (Sec. 8's
mesh density field), the grading, the kinetic-sensor criterion and the state transfer by copy,
uniform explosion and coalescence (Sec. 3.2), checked against identities (a remesh onto the same
map, refinement followed by coarsening), exact conservation of the ledger and a map that reduces
to refinement boxes."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import amr
from oracle import grid as G
from oracle import lattices as L
from oracle import solver as S
from paper_2504_04465_b300 import inputs as I


def disc_map(n, centre, radius, levels):
    x, y = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    r = np.hypot(x - centre[0], y - centre[1])
    return np.where(r < radius, 0, levels - 1).astype(np.uint8)


def _solver(spec, lat, model="rr", seed=9, **kw):
    g = G.build(spec, lat)
    s = S.Solver(g, model, nu0=0.02, **kw)
    fields = []
    for lv in g.levels:
        rho = 1.0 + 0.05 * I.uniform_at(seed, lv.level, lv.coords, 0)
        u = 0.05 * np.stack([I.uniform_at(seed + 1 + k, lv.level, lv.coords, 0) for k in range(lat.D)])
        T = None if model in ("rr", "bgk") else lat.cs2 * (1 + 0.05 * I.uniform_at(seed + 5, lv.level, lv.coords, 0))
        fields.append((rho, u, T))
    s.init_fields(fields)
    return s


def test_level_map_reduces_to_boxes():
    """A map that wants level 0 on a box and level 1 elsewhere builds the box grid."""
    lat = L.D2Q9
    m = np.ones((64, 64), np.uint8)
    m[16:48, 16:48] = 0
    a = G.build(I.GridSpec(2, (64, 64), 2, [], (True, True), level_map=m), lat)
    b = G.build(I.taylor_green_spec(32, 8, 24, 2), lat)
    for la, lb in zip(a.levels, b.levels):
        assert np.array_equal(la.coords, lb.coords) and np.array_equal(la.ctype, lb.ctype)


def test_grading_separates_the_interfaces():
    """After grading, the borders of consecutive regions are at least 3 reach + 1 cells of the
    coarser level apart, and a graded disc builds on every lattice (the builder's ghost-layer
    checks pass)."""
    for name in ("D2Q9", "D2Q21", "D2Q37"):
        lat = L.LATTICES[name]
        m = amr.grade(disc_map(128, (64, 50), 10, 3), 3, lat.reach, (True, True))
        assert m.min() == 0 and m.max() == 2
        G.build(I.GridSpec(2, (128, 128), 3, [], (True, True), level_map=m), lat)
        # level-1 cells (2 finest) around the level-0 footprint: all within region 1
        f0 = np.argwhere(m == 0) // 2
        w = 3 * lat.reach + 1
        for c in f0[:: max(1, len(f0) // 20)]:
            for dx in (-w, w):
                x = ((c[0] + dx) * 2) % 128
                assert m[x, c[1] * 2] <= 1


def test_remesh_onto_the_same_map_is_the_identity():
    lat = L.D2Q9
    m = amr.grade(disc_map(64, (32, 32), 8, 2), 2, lat.reach, (True, True))
    spec = I.GridSpec(2, (64, 64), 2, [], (True, True), level_map=m)
    s = _solver(spec, lat)
    s.step_coarse(3)
    n = amr.remesh(s, spec)
    for lev, lv in enumerate(s.g.levels):
        keep = np.isin(lv.ctype, (G.FLUID, G.BC))
        assert np.array_equal(n.f[lev][:, keep], s.f[lev][:, keep])
    assert np.abs(n.ledger() - s.ledger()).max() < 1e-14 * s.ledger()[0]


def test_refine_then_coarsen_returns_the_state():
    """Uniform explosion followed by coalescence is the identity on the coarse state."""
    lat = L.D2Q21
    coarse = I.GridSpec(2, (128, 128), 2, [], (True, True), level_map=np.ones((128, 128), np.uint8))
    fine_map = amr.grade(disc_map(128, (64, 64), 20, 2), 2, lat.reach, (True, True))
    fine = I.GridSpec(2, (128, 128), 2, [], (True, True), level_map=fine_map)
    s = _solver(coarse, lat)
    s.step_coarse(2)
    back = amr.remesh(amr.remesh(s, fine), coarse)
    assert np.abs(back.f[1] - s.f[1]).max() < 1e-15


@pytest.mark.parametrize("latname,model", [("D2Q9", "rr"), ("D2Q21", "rr"), ("D2Q37", "poly_ddf")])
def test_remesh_keeps_the_ledger(latname, model):
    """Moving a refined disc (refining ahead, coarsening behind) keeps mass, momentum and energy
    of the conserved state exactly (to round-off), and the run goes on conserving them."""
    lat = L.LATTICES[latname]
    kw = {"T0": None} if model == "poly_ddf" else {}
    m1 = amr.grade(disc_map(128, (50, 64), 12, 3), 3, lat.reach, (True, True))
    m2 = amr.grade(disc_map(128, (70, 60), 12, 3), 3, lat.reach, (True, True))
    s = _solver(I.GridSpec(2, (128, 128), 3, [], (True, True), level_map=m1), lat, model)
    s.step_coarse(2)
    l0 = s.ledger()
    n = amr.remesh(s, I.GridSpec(2, (128, 128), 3, [], (True, True), level_map=m2))
    l1 = n.ledger()
    k = lat.D + 1 if model == "rr" else lat.D + 2
    assert np.abs(l1[:k] - l0[:k]).max() < 1e-13 * l0[0]
    n.step_coarse(2)
    assert np.abs(n.ledger()[:k] - l1[:k]).max() < 1e-13 * l0[0] * (1 if model == "rr" else 100)


def test_sensor_flags_the_shock():
    """The kinetic sensor of a Sod tube (D2Q21 numerical equilibrium) exceeds 0.2 only within a
    few cells of the waves; the map refines there and leaves the far field coarse."""
    lat = L.D2Q21
    spec = I.GridSpec(2, (256, 32), 2, [], (True, True), level_map=np.ones((256, 32), np.uint8))
    g = G.build(spec, lat)
    s = S.Solver(g, "num_ddf", nu0=0.0, T0=0.9, sensor_A=1.5)
    lv = g.levels[1]
    c = I.cell_centres(lv.coords, 1)
    rho, u, T = I.sod_fields(c, 256, 0.9)
    rho = np.where(c[:, 0] > 128 + 64, 1.0, rho)           # periodic: one pair of jumps
    s.init_fields([(np.zeros(0), np.zeros((2, 0)), None), (rho, u, np.where(c[:, 0] > 192, 0.9, T))])
    s.step_coarse(4)
    m = amr.sensor_level_map(s, 0.2)
    fine_x = np.unique(np.argwhere(m == 0)[:, 0])
    assert fine_x.size > 0
    assert (m == 1).sum() > 0.5 * m.size
