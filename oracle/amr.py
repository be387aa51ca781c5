"""Adaptive mesh refinement of the oracle: level maps, their grading, the kinetic-sensor
criterion and the transfer of a state onto a rebuilt grid.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sources (arXiv 2504.04465):
  * Sec. 8 (adaptive mesh refinement): a mesh density field gives each cell an integer level
    from 0 (finest) to the tree depth; coarser levels are built around the finer ones with a
    fixed number of cell layers; after the new mesh is set, populations are copied where the
    same cell existed, otherwise rebuilt by coalescence (coarsening) or uniform explosion
    (refinement); the supersonic airfoil flags cells where the kinetic sensor exceeds 0.2.
  * Sec. 3.2, Eqs. coalescence / explosion_uniform (the two transfer rules).
  * Appendix A, Eq. DeltaAvg (the sensor).
Readings (design notes): R39 the density field is given per finest cell and the region of
level i is every level-(i+1) cell holding a finest cell that wants level i or finer; grading
keeps 3 reach + 1 level-(i+1) cells between the borders of regions i and i + 1; R40 the state
carried over is the conserved one (coarse ghosts with their unknowns coalesced, fine ghosts
standing for their coarse-ghost parent), so a transfer keeps the ledger.
"""
from __future__ import annotations

from itertools import product

import numpy as np

from . import hermite as hm
from .grid import BC, CGHOST, FGHOST, FLUID, SOLID, build
from .solver import Solver, sensor_eps


def grade(level_map: np.ndarray, n_levels: int, reach: int, periodic) -> np.ndarray:
    """Return a copy of ``level_map`` in which every level-(i+1) cell within 3 reach + 1
    level-(i+1) cells (Chebyshev) of a level-(i+1) cell holding a finest cell that wants level i
    or finer wants level i + 1 or finer, for i = 0 .. n_levels - 2."""
    m = np.array(level_map, dtype=np.int64)
    width = 3 * reach + 1
    D = m.ndim
    for i in range(n_levels - 1):
        f = 2 ** (i + 1)
        coarse_shape = tuple(e // f for e in m.shape)
        foot = np.zeros(coarse_shape, dtype=bool)
        fine_idx = np.argwhere(m <= i)
        foot[tuple((fine_idx // f).T)] = True
        for ax in range(D):                       # Chebyshev dilation, one axis at a time
            grown = foot.copy()
            for o in range(1, width + 1):
                for sgn in (1, -1):
                    if periodic[ax]:
                        grown |= np.roll(foot, sgn * o, axis=ax)
                    else:
                        sh = np.zeros_like(foot)
                        src = [slice(None)] * D
                        dst = [slice(None)] * D
                        if sgn > 0:
                            src[ax], dst[ax] = slice(0, foot.shape[ax] - o), slice(o, None)
                        else:
                            src[ax], dst[ax] = slice(o, None), slice(0, foot.shape[ax] - o)
                        if foot.shape[ax] > o:
                            sh[tuple(dst)] = foot[tuple(src)]
                        grown |= sh
            foot = grown
        cover = foot
        for ax in range(D):
            cover = np.repeat(cover, f, axis=ax)
        m = np.where(cover & (m > i + 1), i + 1, m)
    return m.astype(np.uint8)


def sensor_level_map(sol: Solver, threshold: float, fixed_map=None) -> np.ndarray:
    """Level map from the kinetic sensor of the pre-collision state (Eq. DeltaAvg): every finest
    cell under a bulk or boundary cell with eps > threshold wants level 0, elsewhere
    ``fixed_map`` (or the coarsest level); then graded."""
    g = sol.g
    L = g.n_levels
    m = np.full(g.extent, L - 1, dtype=np.int64)
    if fixed_map is not None:
        m = np.minimum(m, np.asarray(fixed_map, dtype=np.int64))
    for lev, lv in enumerate(g.levels):
        f = sol.f[lev]
        if sol.comp:
            rho, u, T = sol._moments(f, sol.g_[lev])
            lam0 = sol._guess(u, T, sol.lam[lev]) if sol.lam is not None else None
            feq, _, _ = sol._feq_comp(rho, u, T, lam0)
        else:
            rho, u = hm.macroscopic(sol.lat, f)
            feq = hm.feq_athermal(sol.lat, rho, u)
        eps = sensor_eps(f, feq)
        hit = np.isin(lv.ctype, (FLUID, BC)) & (eps > threshold)
        s = 2 ** lev
        for c in lv.coords[hit]:
            m[tuple(slice(int(x) * s, (int(x) + 1) * s) for x in c)] = 0
    return grade(m, L, sol.lat.reach, g.periodic)


def _lookup(lv, c, periodic):
    c = np.array(c, dtype=np.int64)
    for ax in range(c.size):
        if c[ax] < 0 or c[ax] >= lv.shape[ax]:
            if not periodic[ax]:
                return -1
            c[ax] %= lv.shape[ax]
    return int(lv.index[tuple(c)])


def _sources(g, i, c, w, out):
    """(level, cell, weight) entries of the conserved state a new level-i cell at c takes."""
    lv = g.levels[i]
    k = _lookup(lv, c, g.periodic)
    if k >= 0:
        t = lv.ctype[k]
        if t in (FLUID, BC, CGHOST):
            out.append((i, k, w))
            return
        if t == SOLID:
            return
        if t == FGHOST:                                   # stands for its coarse-ghost parent
            p = _lookup(g.levels[i + 1], [x // 2 for x in c], g.periodic)
            assert p >= 0 and g.levels[i + 1].ctype[p] == CGHOST
            out.append((i + 1, p, w))
            return
    finer = any(_lookup(g.levels[j], [x << (i - j) for x in c], g.periodic) >= 0 for j in range(i))
    if finer:
        kids = list(product((0, 1), repeat=len(c)))       # coalescence of the finer children
        for off in kids:
            _sources(g, i - 1, [2 * x + o for x, o in zip(c, off)], w / len(kids), out)
        return
    for j in range(i + 1, g.n_levels):                    # uniform explosion of a coarser cell
        p = [x >> (j - i) for x in c]
        if _lookup(g.levels[j], p, g.periodic) >= 0:
            _sources(g, j, p, w, out)
            return
    raise ValueError("a new cell has no old state")


def remesh(sol: Solver, spec) -> Solver:
    """A Solver on the grid of ``spec`` (same settings) holding ``sol``'s state carried over: the
    old conserved state per cell (coarse ghosts coalesced), copied, exploded or coalesced."""
    if sol.t % (2 ** (sol.g.n_levels - 1)):
        raise ValueError("remesh at a coarse synchronisation instant only")
    old = sol.g
    state = []                                            # (f, g, lam) per old level
    for lev, lv in enumerate(old.levels):
        f = sol.f[lev].copy()
        gg = sol.g_[lev].copy() if sol.comp else None
        lam = sol.lam[lev].copy() if sol.lam is not None else None
        if lev >= 1 and lv.cg_cells.size:
            cf, cg, cl = sol._coalesced(lev)
            f[:, lv.cg_cells] = cf
            if gg is not None:
                gg[:, lv.cg_cells] = cg
            if lam is not None:
                lam[:, lv.cg_cells] = cl
        state.append((f, gg, lam))
    new_grid = build(spec, sol.lat)
    new = Solver(new_grid, sol.model, nu0=sol.nu[0], T0=sol.T0, gamma=sol.gamma, sensor_A=sol.sensor_A,
                 newton_tol=sol.tol, newton_max_iter=sol.max_iter, guess=sol.guess, poly_order=sol.poly_order,
                 mlp=sol.mlp, trace_eq=sol.trace_eq, trt_magic=sol.trt_magic, sponge=sol.sponge)
    for i, lv in enumerate(new_grid.levels):
        for k in range(lv.n):
            if lv.ctype[k] == SOLID:
                continue
            ent = []
            _sources(old, i, [int(x) for x in lv.coords[k]], 1.0, ent)
            for (j, kk, w) in ent:
                new.f[i][:, k] += w * state[j][0][:, kk]
                if new.comp:
                    new.g_[i][:, k] += w * state[j][1][:, kk]
                if new.lam is not None:
                    new.lam[i][:, k] += w * state[j][2][:, kk]
    # a coarse ghost at a concave corner lets its own streamed population stand in for children
    # whose history leaves the finer level (R33); set those so that its coalesced state is the
    # state carried over (reading R40), which keeps the ledger exact across the remesh
    for lev in range(1, new_grid.n_levels):
        lv = new_grid.levels[lev]
        brk = lv.cg_broken
        if lv.cg_cells.size == 0 or not brk.any():
            continue
        C, kids = lv.cg_cells, lv.cg_children
        nk = kids.shape[1]
        nb = brk.sum(axis=2)                                  # (Q, nc)
        fix = lv.cg_unknown & (nb > 0)
        pops = [(new.f[lev], new.f[lev - 1])] + ([(new.g_[lev], new.g_[lev - 1])] if new.comp else [])
        for coarse, fine in pops:
            v = coarse[:, C]
            kid = fine[:, kids]                               # (Q, nc, nk)
            rest = np.where(brk, 0.0, kid).sum(axis=2)
            own = (nk * v - rest) / np.maximum(nb, 1)
            coarse[:, C] = np.where(fix, own, v)
    new.nonconv = sol.nonconv
    return new
