"""Shared helpers of the parity tests: run the same seeded case through the oracle and through
the CUDA library, and compare them cell by cell (matched by level and coordinates)."""
from __future__ import annotations

import numpy as np

from oracle import grid as G
from oracle import lattices as L
from oracle import solver as S
from paper_2504_04465_b300 import inputs as I

ORACLE_PARAMS = ("nu0", "T0", "gamma", "sensor_A", "newton_tol", "guess", "trace_eq", "trt_magic", "sponge")


def fields_for(lat, fields_fn, level, coords):
    c = I.cell_centres(coords, level)
    out = fields_fn(level, coords, c)
    rho, u = out[0], out[1]
    T = out[2] if len(out) > 2 else None
    return np.asarray(rho, float), np.asarray(u, float).reshape(lat.D, -1), (None if T is None else np.asarray(T, float))


def run_oracle(spec, latname, model, fields_fn, n_fine, **params):
    lat = L.LATTICES[latname]
    g = G.build(spec, lat)
    kw = {k: v for k, v in params.items() if k in ORACLE_PARAMS and v is not None}
    if "T0" in kw and not kw["T0"]:
        kw.pop("T0")
    s = S.Solver(g, model, mlp=params.get("mlp"), **kw)
    s.init_fields([fields_for(lat, fields_fn, lv.level, lv.coords) for lv in g.levels])
    s.step_fine(n_fine)
    return s


def make_gpu(spec, latname, model, storage, fields_fn, block=None, **params):
    from paper_2504_04465_b300 import lbmtree as lt
    lat = L.LATTICES[latname]
    ctx = lt.Context(spec.dim, device=0)
    coll = {k: v for k, v in params.items()
            if k in ORACLE_PARAMS + ("newton_fp32", "newton_max_iter", "streaming") and v is not None}
    ctx.configure(spec, latname, model, storage, block=block, **coll)
    lv, xyz, ty = ctx.cells()
    n = lv.size
    rho = np.ones(n)
    u = np.zeros((spec.dim, n))
    T = np.zeros(n)
    for level in np.unique(lv):
        m = lv == level
        r, uu, tt = fields_for(lat, fields_fn, int(level), xyz[m, :spec.dim])
        rho[m] = r
        u[:, m] = uu
        if tt is not None:
            T[m] = tt
    comp = model in ("poly_ddf", "num_ddf")
    ctx.init_fields(rho, u, T if comp else None)
    return ctx


def gpu_index(ctx, dim):
    lv, xyz, ty = ctx.cells()
    return {(int(l), *map(int, x[:dim])): k for k, (l, x) in enumerate(zip(lv, xyz))}


def matched(sol, ctx, types=(G.FLUID, G.BC)):
    """Triples (oracle level, oracle cell indices, gpu listed indices) for cells of given types."""
    idx = gpu_index(ctx, sol.g.D)
    out = []
    for lev, lv in enumerate(sol.g.levels):
        sel = np.nonzero(np.isin(lv.ctype, types))[0]
        gi = np.array([idx[(lev, *map(int, lv.coords[k]))] for k in sel], dtype=np.int64)
        out.append((lev, sel, gi))
    return out


def rel_l2(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def compare_moments(sol, ctx):
    """Relative L2 of rho, u, T over bulk and boundary cells of every level."""
    rho_g, u_g, T_g = ctx.moments()
    R, U, TT = [], [], []
    for lev, sel, gi in matched(sol, ctx):
        rho_o, u_o, T_o = sol.moments(lev)
        R.append((rho_g[gi], rho_o[sel]))
        U.append((u_g[:, gi], u_o[:, sel]))
        if T_o is not None:
            TT.append((T_g[gi], T_o[sel]))
    out = {
        "rho": rel_l2(np.concatenate([a for a, _ in R]), np.concatenate([b for _, b in R])),
        "u": rel_l2(np.concatenate([a for a, _ in U], axis=1), np.concatenate([b for _, b in U], axis=1)),
    }
    if TT:
        out["T"] = rel_l2(np.concatenate([a for a, _ in TT]), np.concatenate([b for _, b in TT]))
    return out


def near_interface(sol, width=None):
    """Per level, oracle indices of bulk and boundary cells within ``width`` cells (Chebyshev
    distance in the level's own units; default twice the lattice reach) of a coarse ghost, a
    fine ghost or a solid cell: the cells a coupling or bounce-back error reaches first."""
    w = 2 * sol.lat.reach if width is None else width
    out = []
    for lv in sol.g.levels:
        dense = np.zeros(lv.shape, dtype=bool)
        special = np.isin(lv.ctype, (G.CGHOST, G.FGHOST, G.SOLID))
        dense[tuple(lv.coords[special].T)] = True
        near = G._dilate(dense, w, sol.g.periodic)
        hit = near[tuple(lv.coords.T)] & np.isin(lv.ctype, (G.FLUID, G.BC))
        out.append(np.nonzero(hit)[0])
    return out


def compare_near(sol, ctx, width=None):
    """Largest pointwise error of rho, u (every component) and T over the cells of
    ``near_interface``, relative to the largest magnitude of that field over the bulk and
    boundary cells of the whole grid (a level still at rest would otherwise turn rounding noise
    into a large relative error); also the number of cells checked."""
    rho_g, u_g, T_g = ctx.moments()
    idx = gpu_index(ctx, sol.g.D)
    near = near_interface(sol, width)
    scale = {"rho": 0.0, "u": 0.0, "T": 0.0}
    diffs = {"rho": 0.0, "u": 0.0, "T": 0.0}
    worst = {"n": 0}
    for lev, lv in enumerate(sol.g.levels):
        rho_o, u_o, T_o = sol.moments(lev)
        allc = np.nonzero(np.isin(lv.ctype, (G.FLUID, G.BC)))[0]
        if allc.size:
            scale["rho"] = max(scale["rho"], float(np.abs(rho_o[allc]).max()))
            scale["u"] = max(scale["u"], float(np.abs(u_o[:, allc]).max()))
            if T_o is not None:
                scale["T"] = max(scale["T"], float(np.abs(T_o[allc]).max()))
        sel = near[lev]
        if sel.size == 0:
            continue
        gi = np.array([idx[(lev, *map(int, lv.coords[k]))] for k in sel], dtype=np.int64)
        worst["n"] += int(sel.size)
        diffs["rho"] = max(diffs["rho"], float(np.abs(rho_g[gi] - rho_o[sel]).max()))
        diffs["u"] = max(diffs["u"], float(np.abs(u_g[:, gi] - u_o[:, sel]).max()))
        if T_o is not None:
            diffs["T"] = max(diffs["T"], float(np.abs(T_g[gi] - T_o[sel]).max()))
    for k in ("rho", "u", "T"):
        if scale[k] > 0 or k != "T":
            worst[k] = diffs[k] / max(scale[k], 1e-300)
    return worst


# Element-wise bound of FP64 populations for the Newton-solved (numerical) equilibria: both sides
# stop the solve at the first iterate whose largest constraint residual is below 1e-12, and a
# residual right at that threshold can stop one side an iteration earlier than the other, which
# leaves individual populations apart by up to about the tolerance (the moments, averaged over
# the grid, still agree to 1e-15).  Ten times the tolerance.
POP_TOL_NEWTON = 1e-11


def population_map(sol, ctx):
    """perm such that gpu population perm[q] is oracle population q."""
    xi_g = ctx.velocities()[:, : sol.g.D]
    pos = {tuple(int(a) for a in v): k for k, v in enumerate(xi_g)}
    return np.array([pos[tuple(int(a) for a in v)] for v in sol.lat.xi], dtype=np.int64)


def compare_populations(sol, ctx, which="f"):
    """Largest element-wise difference of the populations (f or g) over bulk and boundary
    cells, relative to the largest oracle population of the same level."""
    pops = ctx.populations(which)
    perm = population_map(sol, ctx)
    worst = 0.0
    for lev, sel, gi in matched(sol, ctx):
        if sel.size == 0:
            continue
        o = (sol.f if which == "f" else sol.g_)[lev][:, sel]
        g = pops[perm][:, gi]
        worst = max(worst, float(np.abs(g - o).max() / max(np.abs(o).max(), 1e-300)))
    return worst


def error_curve(spec, latname, model, storage, fields_fn, checkpoints, **params):
    """Step the oracle and the CUDA path side by side and compare them at each checkpoint (fine
    iterations): whole-domain relative L2 (``compare_moments``) and the interface-local relative
    max-abs (``compare_near``, keys prefixed ``near_``).  Returns (oracle, context, curve)."""
    sol = run_oracle(spec, latname, model, fields_fn, 0, **params)
    ctx = make_gpu(spec, latname, model, storage, fields_fn, **params)
    curve, t = [], 0
    for c in checkpoints:
        sol.step_fine(c - t)
        ctx.step_fine(c - t)
        ctx.sync()
        t = c
        e = compare_moments(sol, ctx)
        e.update({"near_" + k: v for k, v in compare_near(sol, ctx).items()})
        curve.append((c, e))
    return sol, ctx, curve


# ------------------------------------------------------------------ seeded initial fields
def tg_fields(coarse_n, n_levels, u0=0.05, cs2=1.0 / 3.0, seed=None, amp=0.0):
    def fn(level, coords, centres):
        rho, u = I.taylor_green_fields(centres, coarse_n, n_levels, u0, cs2)
        if seed is not None:
            u = u + amp * np.stack([I.uniform_at(seed, level, coords, k) for k in range(u.shape[0])])
        return rho, u
    return fn


def smooth_comp_fields(extent, T0, seed=1504):
    ext = np.asarray(extent, float)

    def fn(level, coords, c):
        rho = 1 + 0.1 * np.exp(-((c - ext / 2) ** 2).sum(1) / 64)
        u = np.stack([0.1 + 0 * rho, 0.05 * np.sin(2 * np.pi * c[:, 0] / ext[0])])
        u = u + 0.01 * np.stack([I.uniform_at(seed, level, coords, k) for k in range(2)])
        T = T0 * (1 + 0.05 * np.cos(2 * np.pi * c[:, 1] / ext[1]))
        return rho, u, T
    return fn


def sod_fields(nx, T0):
    def fn(level, coords, c):
        return I.sod_fields(c, nx, T0)
    return fn
