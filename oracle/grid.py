"""Multi-level cell-centred grid with Rohde ghost layers, neighbour lists and boundary cells.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sources (arXiv 2504.04465):
  * Sec. 3.2 and Fig. rohde_highorder: cells of consecutive levels have a 1:2 size ratio; at an
    interface the coarse level keeps `reach` layers of coarse ghost cells inside the refined
    region, overlapping 2*reach layers of fine ghost cells (the children of the coarse ghosts);
    the buffer grows with the lattice size.
  * Sec. 4.3: the parent of overlapping leaves is the (tagged) coarse ghost.
  * Sec. 4.4: every cell stores V-1 neighbour links found by searching the cell at xi_i.
  * Appendix A.3: bounce-back, equilibrium Dirichlet and Neumann conditions applied over as
    many layers as the lattice reach.

Plain construction on dense per-level boolean masks (no blocks, no Morton order -- the order
of cells is irrelevant to the method).  Level 0 is the finest; a level-i cell has edge 2^i in
finest units.  Region_i is the union of the level-i boxes of the spec (the whole domain for
the coarsest level).  Readings used here (design notes): R1 coarse unknowns are the
populations that were not streamed from a coarse bulk cell (no source, or a source that is
itself a coarse ghost) -- the literal "no coarse source" rule loses mass at patch corners,
where diagonal links cut through the fine bulk; R33 at the concave corners of the finer region a
child whose two-step streaming history leaves the finer level enters the coalescence with the
coarse ghost's own streamed population (see ``_coupling``); R11 a link is blocked when
any cell of the lattice segment between the two cells is solid (both roundings taken where
the segment passes between cells); R12 a boundary cell's interior partner is the cell
obtained by clamping its coordinates into the interior along every non-periodic axis.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from itertools import product

import numpy as np

from .lattices import Lattice

FLUID, CGHOST, FGHOST, BC, SOLID = 1, 2, 3, 4, 5
FACES = ["x-", "x+", "y-", "y+", "z-", "z+"]
BC_KINDS = {"dirichlet": 1, "dirichlet_rho": 2, "neumann": 3}
WALL = "wall"     # face kind: halfway bounce-back at the face plane, Ladd's moving-wall term


class GridError(ValueError):
    pass


@dataclass
class Level:
    level: int
    shape: tuple
    coords: np.ndarray            # (n, D) level units
    index: np.ndarray             # dense shape -> cell index or -1
    ctype: np.ndarray             # (n,)
    src: np.ndarray = None        # (Q, n) pull source or -1
    blocked: np.ndarray = None    # (Q, n) bool
    # coupling with the next finer level (level >= 1)
    cg_cells: np.ndarray = None   # (nc,) indices of coarse ghosts
    cg_unknown: np.ndarray = None  # (Q, nc) bool
    cg_children: np.ndarray = None  # (nc, 2^D) indices in the finer level
    cg_broken: np.ndarray = None  # (Q, nc, 2^D) bool: child histories that leave the finer level
    # boundary cells
    bc_cells: np.ndarray = None
    bc_kind: np.ndarray = None
    bc_face: np.ndarray = None
    bc_partner: np.ndarray = None
    wall_term: np.ndarray = None  # (Q, n) velocity term of links bounced at a wall face

    @property
    def n(self) -> int:
        return self.coords.shape[0]


@dataclass
class Grid:
    lat: Lattice
    D: int
    extent: tuple
    n_levels: int
    periodic: tuple
    faces: dict
    levels: list = field(default_factory=list)

    def n_eq(self) -> float:
        """Equivalent fine cells N_eq = sum_i n_i / 2^i over non-solid cells (Sec. 7.5)."""
        return sum(float((lv.ctype != SOLID).sum()) / 2 ** lv.level for lv in self.levels)


# ----------------------------------------------------------------------------- helpers
def _dilate(mask: np.ndarray, r: int, periodic) -> np.ndarray:
    out = mask.copy()
    D = mask.ndim
    for off in product(range(-r, r + 1), repeat=D):
        if not any(off):
            continue
        out |= _shift(mask, off, periodic)
    return out


def _shift(mask: np.ndarray, off, periodic) -> np.ndarray:
    """result[x] = mask[x - off] (False outside non-periodic bounds)."""
    res = mask
    for ax, o in enumerate(off):
        if o == 0:
            continue
        if periodic[ax]:
            res = np.roll(res, o, axis=ax)
        else:
            tmp = np.zeros_like(res)
            n = res.shape[ax]
            sl_dst = [slice(None)] * res.ndim
            sl_src = [slice(None)] * res.ndim
            if o > 0:
                sl_dst[ax] = slice(o, n)
                sl_src[ax] = slice(0, n - o)
            else:
                sl_dst[ax] = slice(0, n + o)
                sl_src[ax] = slice(-o, n)
            tmp[tuple(sl_dst)] = res[tuple(sl_src)]
            res = tmp
    return res


def _block_min(a: np.ndarray, f: int) -> np.ndarray:
    """Minimum over blocks of f cells per axis."""
    for ax in range(a.ndim):
        sh = list(a.shape)
        sh[ax:ax + 1] = [sh[ax] // f, f]
        a = a.reshape(sh).min(axis=ax + 1)
    return a


def _region_mask(spec, level: int, shape) -> np.ndarray:
    """Region_level at level resolution: the union of that level's boxes, or, from a level map
    (the finest level wanted at each finest cell, Sec. 8's mesh density field), every cell whose
    parent holds a finest cell wanting this level or finer (aligned to parents by construction)."""
    if level >= spec.n_levels - 1:
        return np.ones(shape, dtype=bool)
    lmap = getattr(spec, "level_map", None)
    if lmap is not None:
        if spec.boxes:
            raise GridError("give refinement boxes or a level map, not both")
        lmap = np.asarray(lmap)
        if lmap.shape != tuple(spec.extent) or lmap.max() >= spec.n_levels or lmap.min() < 0:
            raise GridError("level map of the wrong shape or with entries beyond the coarsest level")
        parent = _block_min(lmap, 2 ** (level + 1)) <= level
        for ax in range(parent.ndim):
            parent = np.repeat(parent, 2, axis=ax)
        return parent
    m = np.zeros(shape, dtype=bool)
    s = 2 ** level
    for (lv, lo, hi) in spec.boxes:
        if lv != level:
            continue
        sl = []
        for d in range(len(shape)):
            if lo[d] % (2 * s) or hi[d] % (2 * s):
                raise GridError(f"box of level {lv} not aligned to {2 * s}")
            sl.append(slice(lo[d] // s, hi[d] // s))
        m[tuple(sl)] = True
    return m


def _coarsen(mask_fine: np.ndarray) -> np.ndarray:
    """Level-(i+1) cell is inside iff all its children are."""
    D = mask_fine.ndim
    out = None
    for off in product((0, 1), repeat=D):
        sl = tuple(slice(o, None, 2) for o in off)
        out = mask_fine[sl] if out is None else (out & mask_fine[sl])
    return out


def _refine(mask_coarse: np.ndarray) -> np.ndarray:
    out = mask_coarse
    for ax in range(mask_coarse.ndim):
        out = np.repeat(out, 2, axis=ax)
    return out


def solid_mask_level0(spec, shape) -> np.ndarray:
    """Cells of level 0 whose centre lies inside one of the analytic shapes."""
    D = len(shape)
    centres = np.meshgrid(*[np.arange(n) + 0.5 for n in shape], indexing="ij")
    m = np.zeros(shape, dtype=bool)
    for s in getattr(spec, "solids", []) or []:
        if s["kind"] == "sphere":
            r2 = sum((centres[d] - s["center"][d]) ** 2 for d in range(D))
            m |= r2 < s["radius"] ** 2
        elif s["kind"] == "naca":
            # symmetric NACA 4-digit thickness, closed trailing edge, zero angle of attack
            c, t = s["chord"], s.get("t", 0.12)
            xr = (centres[0] - s["x0"]) / c
            inside_x = (xr >= 0.0) & (xr <= 1.0)
            xc = np.clip(xr, 0.0, 1.0)
            yt = 5.0 * t * c * (0.2969 * np.sqrt(xc) - 0.1260 * xc - 0.3516 * xc ** 2
                                + 0.2843 * xc ** 3 - 0.1036 * xc ** 4)
            m |= inside_x & (np.abs(centres[1] - s["y0"]) < yt)
        elif s["kind"] == "mask":
            m |= np.asarray(s["mask"], dtype=bool)
        else:
            raise GridError(f"unknown solid kind {s['kind']}")
    return m


def _segment_cells(xi) -> list:
    """Offsets o (to subtract from x) of the cells met on the segment x -> x - xi (R11)."""
    n = int(max(abs(int(v)) for v in xi))
    cells = set()
    for m in range(1, n + 1):
        opts = []
        for v in xi:
            p = m * int(v) / n
            lo, hi = int(np.floor(p)), int(np.ceil(p))
            opts.append({lo, hi})
        for o in product(*opts):
            cells.add(tuple(o))
    return sorted(cells)


# ----------------------------------------------------------------------------- builder
def build(spec, lat: Lattice) -> Grid:
    D = spec.dim
    L = spec.n_levels
    reach = lat.reach
    periodic = tuple(spec.periodic)
    g = Grid(lat, D, tuple(spec.extent), L, periodic, dict(getattr(spec, "faces", {}) or {}))
    shapes = []
    for i in range(L):
        if any(e % (2 ** i) for e in spec.extent):
            raise GridError("extent not divisible by 2^(levels-1)")
        shapes.append(tuple(e // 2 ** i for e in spec.extent))
    regions = [_region_mask(spec, i, shapes[i]) for i in range(L)]
    # nesting: Region_{i-1} inside Region_i
    for i in range(1, L):
        if (_coarsen(regions[i - 1]) & ~regions[i]).any():
            raise GridError(f"region {i - 1} not nested in region {i}")
    # cell sets
    bulk, cghost, cells = [], [], []
    for i in range(L):
        finer = _coarsen(regions[i - 1]) if i >= 1 else np.zeros(shapes[i], bool)
        b = regions[i] & ~finer
        cg = finer & _dilate(b, reach, periodic) if i >= 1 else np.zeros(shapes[i], bool)
        bulk.append(b)
        cghost.append(cg)
        cells.append(b | cg)
    solid0 = solid_mask_level0(spec, shapes[0]) & cells[0]
    for i in range(L):
        shape = shapes[i]
        ct = np.zeros(shape, dtype=np.uint8)
        ct[cells[i]] = FLUID
        ct[cghost[i]] = CGHOST
        if i + 1 < L:
            fg = _refine(cghost[i + 1])
            if (fg & ~bulk[i]).any():
                raise GridError(f"fine ghosts of level {i} overlap another ghost layer")
            ct[fg] = FGHOST
            if (_dilate(fg, reach, periodic) & cghost[i]).any():
                raise GridError(f"ghost layers of level {i} closer than the lattice reach")
        if i == 0:
            ct[solid0] = SOLID
        # boundary layers on non-periodic faces
        bc_face = np.full(shape, -1, dtype=np.int64)
        for ax in range(D):
            if periodic[ax]:
                continue
            idx = np.arange(shape[ax])
            for side, sel in ((0, idx < reach), (1, idx >= shape[ax] - reach)):
                face = 2 * ax + side
                bshape = [1] * D
                bshape[ax] = shape[ax]
                layer = np.broadcast_to(sel.reshape(bshape), shape) & cells[i]
                if FACES[face] not in g.faces:
                    raise GridError(f"non-periodic face {FACES[face]} has no boundary condition")
                if g.faces[FACES[face]][0] == WALL:
                    # a wall face has no boundary layer; its links bounce back (_links).  Ghost
                    # layers within the reach of a wall would need bounce-back in pure-streaming
                    # cells, which the method does not define: refused
                    near = np.broadcast_to(sel.reshape(bshape), shape)
                    if (near & ((ct == CGHOST) | (ct == FGHOST))).any():
                        raise GridError(f"ghost layers of level {i} within the reach of wall face {FACES[face]}")
                    continue
                # priority: any Dirichlet face over Neumann; among equals, the first face
                kind = BC_KINDS[g.faces[FACES[face]][0]]
                cur = bc_face >= 0
                cur_kind = np.zeros(shape, dtype=np.int64)
                cur_kind[cur] = [BC_KINDS[g.faces[FACES[f]][0]] for f in bc_face[cur]]
                take = layer & ((~cur) | ((kind != 3) & (cur_kind == 3)))
                bc_face[take] = face
        isbc = bc_face >= 0
        if (isbc & (ct != FLUID)).any():
            raise GridError(f"boundary layers of level {i} touch a ghost or solid cell")
        ct[isbc] = BC
        if i == 0 and solid0.any():
            near = _dilate(solid0, reach, periodic)
            if (near & ((ct == FGHOST) | (ct == BC))).any():
                raise GridError("solid closer than the lattice reach to a ghost or boundary layer")
        coords = np.argwhere(ct > 0)
        index = np.full(shape, -1, dtype=np.int64)
        index[tuple(coords.T)] = np.arange(coords.shape[0])
        lv = Level(i, shape, coords, index, ct[tuple(coords.T)].copy())
        lv.bc_cells = index[tuple(np.argwhere(isbc).T)]
        lv.bc_face = bc_face[tuple(coords[lv.bc_cells].T)] if lv.bc_cells.size else np.zeros(0, np.int64)
        lv.bc_kind = np.array([BC_KINDS[g.faces[FACES[f]][0]] for f in lv.bc_face], dtype=np.int64)
        g.levels.append(lv)
    for i in range(L):
        _links(g, i, solid0 if i == 0 else None)
    for i in range(1, L):
        _coupling(g, i)
    for i in range(L):
        _bc_partners(g, i)
    return g


def _links(g: Grid, i: int, solid0) -> None:
    lv = g.levels[i]
    lat = g.lat
    Q, n = lat.Q, lv.n
    shape = np.array(lv.shape)
    src = np.full((Q, n), -1, dtype=np.int64)
    blocked = np.zeros((Q, n), dtype=bool)
    solid_cells = lv.ctype == SOLID
    for q in range(Q):
        s = lv.coords - lat.xi[q][None, :]
        ok = np.ones(n, dtype=bool)
        for ax in range(g.D):
            if g.periodic[ax]:
                s[:, ax] %= shape[ax]
            else:
                ok &= (s[:, ax] >= 0) & (s[:, ax] < shape[ax])
        idx = np.full(n, -1, dtype=np.int64)
        idx[ok] = lv.index[tuple(s[ok].T)]
        src[q] = idx
        if solid0 is not None and solid0.any() and any(lat.xi[q]):
            for off in _segment_cells(lat.xi[q]):
                c = lv.coords - np.array(off)[None, :]
                okc = np.ones(n, dtype=bool)
                for ax in range(g.D):
                    if g.periodic[ax]:
                        c[:, ax] %= shape[ax]
                    else:
                        okc &= (c[:, ax] >= 0) & (c[:, ax] < shape[ax])
                hit = np.zeros(n, dtype=bool)
                hit[okc] = solid0[tuple(c[okc].T)]
                blocked[q] |= hit
    # wall faces (Appendix A.3, Ladd's velocity bounce-back): a link whose source lies outside
    # the domain through wall faces only bounces back and gains 2 w_q (xi_q . rho_w u_w) / c_s^2,
    # with rho_w u_w the mean over the faces the link crosses (reading R38)
    wall_term = np.zeros((Q, n))
    for q in range(Q):
        s = lv.coords - lat.xi[q][None, :]
        crossed = np.zeros(n, dtype=np.int64)
        nonwall = np.zeros(n, dtype=bool)
        mom = np.zeros((n, g.D))
        for ax in range(g.D):
            if g.periodic[ax]:
                continue
            for side, out in ((0, s[:, ax] < 0), (1, s[:, ax] >= shape[ax])):
                if not out.any():
                    continue
                spec_f = g.faces.get(FACES[2 * ax + side])
                if spec_f is None or spec_f[0] != WALL:
                    nonwall |= out
                    continue
                rho_w = spec_f[1] if len(spec_f) > 1 else 1.0
                u_w = np.asarray(spec_f[2] if len(spec_f) > 2 else (0.0,) * 3, float)[: g.D]
                crossed += out
                mom[out] += rho_w * u_w[None, :]
        wall = (crossed > 0) & ~nonwall & (src[q] < 0)
        blocked[q] |= wall
        if wall.any():
            mean = mom[wall] / crossed[wall][:, None]
            wall_term[q, wall] = 2.0 * lat.w[q] * (mean @ lat.xi[q].astype(np.float64)) / lat.cs2
    blocked[:, solid_cells] = False
    wall_term[:, solid_cells] = 0.0
    lv.src, lv.blocked, lv.wall_term = src, blocked, wall_term
    # every bulk fluid cell must see a cell (or a solid) in every direction
    fl = lv.ctype == FLUID
    missing = (src < 0) & ~blocked & fl[None, :]
    if missing.any():
        raise GridError(f"fluid cells of level {i} with missing neighbours (region touches a face?)")


def _coupling(g: Grid, i: int) -> None:
    lv, fine = g.levels[i], g.levels[i - 1]
    cg = np.nonzero(lv.ctype == CGHOST)[0]
    lv.cg_cells = cg
    # a coarse-ghost population is coalesced unless it was streamed from a coarse bulk
    # (fluid or boundary) cell: populations arriving from another coarse ghost or from the
    # region covered by the finer level are supplied by the finer level (reading R1)
    # (the rest population stays in its own cell and is always known)
    s = lv.src[:, cg]
    from_bulk = np.zeros(s.shape, dtype=bool)
    ok = s >= 0
    from_bulk[ok] = np.isin(lv.ctype[s[ok]], (FLUID, BC))
    rest = ~np.any(g.lat.xi != 0, axis=1)
    from_bulk[rest, :] = True
    lv.cg_unknown = ~from_bulk
    kids = []
    for off in product((0, 1), repeat=g.D):
        c = 2 * lv.coords[cg] + np.array(off)[None, :]
        kids.append(fine.index[tuple(c.T)])
    lv.cg_children = np.stack(kids, axis=1) if cg.size else np.zeros((0, 2 ** g.D), np.int64)
    if (lv.cg_children < 0).any():
        raise GridError("coarse ghost without its fine children")
    if cg.size and not (fine.ctype[lv.cg_children] == FGHOST).all():
        raise GridError("children of a coarse ghost are not fine ghosts")
    # reading R33 (concave corners of the finer region): over one coarse step a fine ghost only
    # streams, so a child's population q at the coalescence left the fine cell ch - 2 xi_q two
    # fine iterations earlier through ch - xi_q.  Where that history leaves the finer level
    # (ch - xi_q is no fine cell, or is a fine ghost and ch - 2 xi_q is none) the packet came
    # from the coarse side and is the coarse ghost's own streamed population instead (the
    # post-collision population of ch's coarse cell minus xi_q, which is the coarse cell
    # holding ch - 2 xi_q).  Only unknown populations are marked; along straight interfaces and
    # at convex corners no history leaves the finer level.
    nk = lv.cg_children.shape[1]
    brk = np.zeros((g.lat.Q, cg.size, nk), dtype=bool)
    for k in range(nk):
        ch = fine.coords[lv.cg_children[:, k]]
        for q in range(g.lat.Q):
            xi = g.lat.xi[q][None, :]
            if not xi.any():
                continue
            i1 = _lookup(fine, ch - xi, g.periodic)
            i2 = _lookup(fine, ch - 2 * xi, g.periodic)
            t1 = np.where(i1 >= 0, fine.ctype[np.maximum(i1, 0)], 0)
            brk[q, :, k] = (i1 < 0) | ((t1 == FGHOST) & (i2 < 0))
    brk &= lv.cg_unknown[:, :, None]
    if (brk.any(axis=2) & (s < 0)).any():
        raise GridError("a coarse ghost stands in for a fine history but has no coarse source")
    lv.cg_broken = brk


def _lookup(lv: Level, c: np.ndarray, periodic) -> np.ndarray:
    """Index of the cell of ``lv`` at level coordinates c (wrapped across periodic faces), -1 where
    there is none."""
    c = c.copy()
    ok = np.ones(c.shape[0], dtype=bool)
    for ax in range(c.shape[1]):
        if periodic[ax]:
            c[:, ax] %= lv.shape[ax]
        else:
            ok &= (c[:, ax] >= 0) & (c[:, ax] < lv.shape[ax])
    out = np.full(c.shape[0], -1, dtype=np.int64)
    out[ok] = lv.index[tuple(c[ok].T)]
    return out


def _bc_partners(g: Grid, i: int) -> None:
    lv = g.levels[i]
    reach = g.lat.reach
    if lv.bc_cells is None or lv.bc_cells.size == 0:
        lv.bc_partner = np.zeros(0, dtype=np.int64)
        return
    c = lv.coords[lv.bc_cells].copy()
    for ax in range(g.D):
        if not g.periodic[ax]:
            c[:, ax] = np.clip(c[:, ax], reach, lv.shape[ax] - 1 - reach)
    p = lv.index[tuple(c.T)]
    if (p < 0).any() or (lv.ctype[p] == BC).any():
        raise GridError("boundary cell without an interior partner")
    lv.bc_partner = p
