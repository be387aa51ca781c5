"""Pins of the oracle's grid builder: hand counts of the ghost layers and link rules."""
import numpy as np
import pytest

from oracle import grid as G
from oracle import lattices as L
from paper_2504_04465_b300 import inputs as I


def test_two_level_taylor_green_counts():
    # 64x64 coarse, central 32x32-coarse patch: 64^2 - 32^2 coarse bulk, a 1-cell coarse ghost
    # ring (32^2 - 30^2), a 64x64 fine patch whose outer 2 rings are fine ghosts (64^2 - 60^2)
    g = G.build(I.taylor_green_spec(64, 16, 48, 2), L.D2Q9)
    c, f = g.levels[1], g.levels[0]
    assert (c.ctype == G.FLUID).sum() == 64 * 64 - 32 * 32
    assert (c.ctype == G.CGHOST).sum() == 32 * 32 - 30 * 30
    assert f.n == 64 * 64
    assert (f.ctype == G.FGHOST).sum() == 64 * 64 - 60 * 60
    assert g.n_eq() == pytest.approx(4096 + (3072 + 124) / 2)
    # every coarse ghost has 4 fine-ghost children
    assert c.cg_children.shape == (124, 4)


def test_reach3_ghost_thickness():
    lat = L.D2Q21
    g = G.build(I.GridSpec(2, (128, 128), 2, [(0, (32, 32), (96, 96))], (True, True)), lat)
    c, f = g.levels[1], g.levels[0]
    assert (c.ctype == G.CGHOST).sum() == 32 * 32 - 26 * 26        # 3 coarse layers
    assert (f.ctype == G.FGHOST).sum() == 64 * 64 - 52 * 52        # 6 fine layers


def test_corner_unknowns():
    # at a convex patch corner only the population arriving from the fine bulk diagonal is
    # unknown; along an edge the three populations coming from the fine side plus the two
    # populations streamed along the ghost strip from neighbouring ghosts
    lat = L.D2Q9
    g = G.build(I.taylor_green_spec(16, 4, 12, 2), lat)
    c = g.levels[1]
    row = {tuple(x): k for k, x in enumerate(c.coords[c.cg_cells])}
    corner = row[(4, 4)]
    unk = {tuple(lat.xi[q]) for q in range(lat.Q) if c.cg_unknown[q, corner]}
    # sources of (4,4): bulk at x<4 or y<4; ghost strip cells (5,4),(4,5),(5,5)->fine bulk
    assert unk == {(-1, -1), (-1, 0), (0, -1)}
    edge = row[(4, 8)]
    unk = {tuple(lat.xi[q]) for q in range(lat.Q) if c.cg_unknown[q, edge]}
    assert unk == {(-1, -1), (-1, 0), (-1, 1), (0, 1), (0, -1)}


def test_segment_cells_symmetric():
    for v in [(3, 1), (2, 1), (3, 0), (2, 2), (1, 1)]:
        fwd = {tuple(o) for o in G._segment_cells(v)}
        back = {tuple(np.array(v) - np.array(o)) for o in G._segment_cells(v)}
        assert fwd | {(0, 0)} == back | {(0, 0)} or fwd - {tuple(v)} == back - {(0, 0)}
        assert tuple(v) in fwd


def test_bounce_back_links_around_solid():
    lat = L.D2Q9
    spec = I.GridSpec(2, (16, 16), 1, [], (True, True), solids=[{"kind": "sphere", "center": (8.0, 8.0), "radius": 2.1}])
    g = G.build(spec, lat)
    lv = g.levels[0]
    solid = lv.ctype == G.SOLID
    for q in range(lat.Q):
        src = lv.src[q]
        fl = ~solid
        assert np.array_equal(lv.blocked[q, fl], solid[src[fl]])


def test_bad_specs_rejected():
    lat = L.D2Q9
    with pytest.raises(G.GridError):          # box touching a non-periodic face
        G.build(I.GridSpec(2, (64, 64), 2, [(0, (0, 16), (32, 48))], (False, True),
                           {"x-": ("neumann",), "x+": ("neumann",)}), lat)
    with pytest.raises(G.GridError):          # nested levels too close
        G.build(I.GridSpec(2, (128, 128), 3, [(1, (32, 32), (96, 96)), (0, (36, 36), (92, 92))],
                           (True, True)), lat)
    with pytest.raises(G.GridError):          # misaligned box
        G.build(I.GridSpec(2, (64, 64), 2, [(0, (15, 16), (48, 48))], (True, True)), lat)
