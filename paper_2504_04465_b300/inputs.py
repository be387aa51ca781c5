"""Seeded synthetic workloads: grid specifications and initial macroscopic fields.

This module holds no arithmetic of the method itself.  It describes grids (extent, refinement
boxes, periodic axes, boundary faces, analytic solids) and evaluates initial fields (density,
velocity, temperature) at cell-centre positions.  Both the CUDA path and the CPU oracle receive
the same arrays from here; neither re-implements a random generator.

Positions are in finest-level units; a level-i cell with integer coordinates c has its centre
at (c + 1/2) * 2^i.  Random perturbations use splitmix64 (Steele, Lea & Flood, OOPSLA 2014)
keyed by (seed, level, cell coordinates), so a cell's value does not depend on the order in
which a caller lists cells.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class GridSpec:
    dim: int
    extent: tuple                       # finest units
    n_levels: int
    boxes: list = field(default_factory=list)   # (level, lo, hi) finest units, level < n_levels-1
    periodic: tuple = (True, True, True)
    faces: dict = field(default_factory=dict)   # face -> (kind, rho, (ux, uy, uz), T)
    solids: list = field(default_factory=list)  # dicts: sphere / naca
    # instead of boxes: the finest level wanted at each finest cell, an integer array of shape
    # extent (0 finest .. n_levels - 1 coarsest)
    level_map: object = None


def cell_centres(coords: np.ndarray, level) -> np.ndarray:
    """Centres in finest units of level cells with integer coords (n, D)."""
    s = (2.0 ** np.asarray(level, dtype=np.float64))
    if np.ndim(s):
        s = s[:, None]
    return (np.asarray(coords, dtype=np.float64) + 0.5) * s


# ------------------------------------------------------------------ counter-based uniforms
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniform_at(seed: int, level, coords: np.ndarray, stream: int) -> np.ndarray:
    """U(-1, 1) per cell, a pure function of (seed, level, coords, stream)."""
    coords = np.asarray(coords, dtype=np.int64)
    n, D = coords.shape
    with np.errstate(over="ignore"):
        key = _splitmix64(np.full(n, np.uint64(seed) * np.uint64(0x100000001B3) + np.uint64(stream), dtype=np.uint64))
        key = _splitmix64(key ^ np.asarray(level, dtype=np.uint64))
        for d in range(D):
            key = _splitmix64(key ^ coords[:, d].astype(np.uint64))
    return (key >> np.uint64(11)).astype(np.float64) * (2.0 / 2.0 ** 53) - 1.0


# ------------------------------------------------------------------ Taylor-Green (2D periodic)
def taylor_green_spec(coarse_n: int = 64, patch_lo: int = 16, patch_hi: int = 48, n_levels: int = 2) -> GridSpec:
    """Periodic square of coarse_n^2 coarse cells with a central patch refined once."""
    s = 2 ** (n_levels - 1)
    ext = (coarse_n * s, coarse_n * s)
    boxes = []
    if patch_hi > patch_lo:
        boxes.append((n_levels - 2, (patch_lo * s, patch_lo * s), (patch_hi * s, patch_hi * s)))
    return GridSpec(2, ext, n_levels, boxes, (True, True))


def taylor_green_fields(centres: np.ndarray, coarse_n: int, n_levels: int, u0: float, cs2: float, rho0: float = 1.0):
    """u_x = -u0 cos(kx) sin(ky), u_y = u0 sin(kx) cos(ky), rho = rho0 + p/c_s^2,
    p = -rho0 u0^2/4 (cos 2kx + cos 2ky), k = 2 pi / coarse_n in coarse units."""
    s = 2.0 ** (n_levels - 1)
    x = centres[:, 0] / s
    y = centres[:, 1] / s
    k = 2.0 * np.pi / coarse_n
    ux = -u0 * np.cos(k * x) * np.sin(k * y)
    uy = u0 * np.sin(k * x) * np.cos(k * y)
    p = -rho0 * u0 ** 2 / 4.0 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    rho = rho0 + p / cs2
    return rho, np.stack([ux, uy])


# ------------------------------------------------------------------ acoustic pulse
def gaussian_pulse_fields(centres: np.ndarray, centre, amp: float, width: float, rho0: float = 1.0):
    r2 = ((centres - np.asarray(centre)[None, :]) ** 2).sum(axis=1)
    rho = rho0 * (1.0 + amp * np.exp(-r2 / width ** 2))
    return rho, np.zeros((centres.shape[1], centres.shape[0]))


# ------------------------------------------------------------------ Sod shock tube
SOD_LEFT = (1.0, 1.0)      # (rho, p) left of the membrane
SOD_RIGHT = (0.125, 0.1)   # (rho, p) right of the membrane


def sod_spec(nx: int, ny: int, n_levels: int = 1, band: tuple | None = None) -> GridSpec:
    """Tube along x: Neumann faces at x = 0 and x = nx, periodic in y.

    ``band`` = (x_lo, x_hi) in finest units: with two levels, the full-height band is the
    finest level and the rest of the tube the coarse one."""
    boxes = []
    if band is not None:
        if n_levels != 2:
            raise ValueError("a refined band needs exactly two levels")
        boxes.append((0, (band[0], 0), (band[1], ny)))
    faces = {"x-": ("neumann",), "x+": ("neumann",)}
    return GridSpec(2, (nx, ny), n_levels, boxes, (False, True), faces)


def sod_fields(centres: np.ndarray, nx: int, T0: float):
    """rho, u = 0, T = T0 p / rho with the classic Sod states (membrane at nx / 2)."""
    left = centres[:, 0] < nx / 2
    rho = np.where(left, SOD_LEFT[0], SOD_RIGHT[0])
    p = np.where(left, SOD_LEFT[1], SOD_RIGHT[1])
    return rho, np.zeros((2, rho.size)), T0 * p / rho


# ------------------------------------------------------------------ 2D Riemann problem, configuration 12
# Quadrant states of Sec. 6.2 (rho / rho0, u_x / u0, u_y / u0, p / p0), quadrants numbered
# counter-clockwise from x > 0, y > 0; u0 = sqrt(gamma T0), p0 = rho0 T0, rho0 = 1.
RIEMANN12 = {1: (0.513, 0.0, 0.0, 0.4), 2: (1.0, 0.7276, 0.0, 1.0), 3: (0.8, 0.0, 0.0, 1.0), 4: (1.0, 0.0, 0.7276, 1.0)}


def riemann12_spec(nc: int, grid: str) -> GridSpec:
    """The [-L, L]^2 domain of the 2D Riemann problem with N_c = nc coarse cells per L (2 nc per
    side), two levels, periodic on every face, refined on one of the grids of Sec. 6.2:
      diag   the half x > y (finest-level box per coarse row: a staircase along the diagonal, whose
             interface is the symmetry line of the initial state);
      axes   bands |x| < L/4 and |y| < L/4 along both axes;
      optim  the axes bands and the central square |x|, |y| < L/2.
    Positions in finest units: the domain is [0, 4 nc)^2 with its centre at 2 nc."""
    ext = 4 * nc
    c = 2 * nc
    boxes = []
    if grid == "diag":
        for j in range(2 * nc - 1):            # coarse row j: coarse cells i > j refined
            boxes.append((0, (2 * (j + 1), 2 * j), (ext, 2 * j + 2)))
    elif grid in ("axes", "optim"):
        w = nc // 2                             # L/4 in finest units (L = 2 nc)
        boxes += [(0, (c - w, 0), (c + w, ext)), (0, (0, c - w), (ext, c + w))]
        if grid == "optim":
            boxes.append((0, (c - nc, c - nc), (c + nc, c + nc)))
    elif grid != "uniform":
        raise ValueError(grid)
    return GridSpec(2, (ext, ext), 2 if boxes else 1, boxes, (True, True))


def riemann12_fields(centres: np.ndarray, nc: int, T0: float, gamma: float = 1.4):
    """rho, u, T of configuration 12 at cell centres (finest units): T = T0 (p/p0) / (rho/rho0)."""
    c = 2 * nc
    x = centres[:, 0] - c
    y = centres[:, 1] - c
    q = np.where(x > 0, np.where(y > 0, 1, 4), np.where(y > 0, 2, 3))
    tab = np.array([RIEMANN12[k] for k in (1, 2, 3, 4)])
    st = tab[q - 1]
    u0 = np.sqrt(gamma * T0)
    rho = st[:, 0]
    u = np.stack([st[:, 1] * u0, st[:, 2] * u0])
    return rho, u, T0 * st[:, 3] / rho


# ------------------------------------------------------------------ lid-driven cavity
def cavity_spec(n: int, lid_u: float, n_levels: int = 1, patch: tuple | None = None, dim: int = 2) -> GridSpec:
    """The L x L (x L) lid-driven cavity of Sec. 5.1 in finest units (n cells per side): wall faces
    (halfway bounce-back) on every side, the lid y+ moving along x at lid_u (Ladd's velocity
    bounce-back, Appendix A.3).  patch = (lo, hi): a centred refinement box (finest units, on
    every axis) kept at least the lattice reach from the walls."""
    faces = {f: ("wall", 1.0, (0.0, 0.0, 0.0)) for f in ("x-", "x+", "y-", "y+", "z-", "z+")[: 2 * dim]}
    faces["y+"] = ("wall", 1.0, (lid_u, 0.0, 0.0))
    boxes = []
    if patch is not None:
        lo, hi = patch
        boxes.append((0, (lo,) * dim, (hi,) * dim))
    return GridSpec(dim, (n,) * dim, n_levels, boxes, (False,) * dim, faces)


def couette_spec(nx: int, ny: int, wall_u: float) -> GridSpec:
    """Plane Couette flow: periodic along x, a resting wall at y- and a wall moving along x at
    y+ (finest units, one level)."""
    faces = {"y-": ("wall", 1.0, (0.0, 0.0, 0.0)), "y+": ("wall", 1.0, (wall_u, 0.0, 0.0))}
    return GridSpec(2, (nx, ny), 1, [], (True, False), faces)


# ------------------------------------------------------------------ 3D flow past a sphere
def sphere_spec(scale: int = 1) -> GridSpec:
    """Four-level box around a sphere: 1024x512x512 finest units at scale 1, sphere diameter 64
    centred at (256, 256, 256); uniform inflow at x-, Neumann on the other faces.

    Level boxes (finest units, scale 1): L0 x[160,672) y,z[128,384); L1 x[96,864) y,z[64,448);
    L2 x[32,992) y,z[32,480); L3 the rest.  scale = 2 halves every extent (the profiling case);
    scale = 4 gives the reduced copy (256x128x128,
    sphere diameter 16) whose boxes keep every ghost layer at least the lattice reach away from
    the next one: L0 x[48,176) y,z[40,88); L1 x[32,224) y,z[32,96); L2 x[16,240) y,z[16,112).
    """
    if scale == 1:
        ext = (1024, 512, 512)
        boxes = [(2, (32, 32, 32), (992, 480, 480)), (1, (96, 64, 64), (864, 448, 448)),
                 (0, (160, 128, 128), (672, 384, 384))]
        centre, radius = (256.0, 256.0, 256.0), 32.0
    elif scale == 2:
        ext = (512, 256, 256)
        boxes = [(2, (16, 16, 16), (496, 240, 240)), (1, (48, 32, 32), (432, 224, 224)),
                 (0, (80, 64, 64), (336, 192, 192))]
        centre, radius = (128.0, 128.0, 128.0), 16.0
    elif scale == 4:
        ext = (256, 128, 128)
        boxes = [(2, (16, 16, 16), (240, 112, 112)), (1, (32, 32, 32), (224, 96, 96)),
                 (0, (48, 40, 40), (176, 88, 88))]
        centre, radius = (64.0, 64.0, 64.0), 8.0
    else:
        raise ValueError("scale must be 1, 2 or 4")
    u_in = SPHERE_MACH / np.sqrt(3.0)
    faces = {"x-": ("dirichlet_rho", 1.0, (u_in, 0.0, 0.0)), "x+": ("neumann",),
             "y-": ("neumann",), "y+": ("neumann",), "z-": ("neumann",), "z+": ("neumann",)}
    return GridSpec(3, ext, 4, boxes, (False, False, False), faces,
                    [{"kind": "sphere", "center": centre, "radius": radius}])


SPHERE_MACH = 0.1
SPHERE_RE = 3900.0
SPHERE_SEED = 3900


def sphere_nu0(scale: int = 1) -> float:
    """Level-0 viscosity u D / Re with D the sphere diameter in finest cells."""
    return SPHERE_MACH / np.sqrt(3.0) * (64.0 / scale) / SPHERE_RE


def sphere_fields(level, coords: np.ndarray):
    """rho = 1, u = u_inf (1, 0, 0) + 1e-3 u_inf U(-1, 1)^3 per cell (splitmix64, seed 3900)."""
    coords = np.asarray(coords)
    n = coords.shape[0]
    u_in = SPHERE_MACH / np.sqrt(3.0)
    u = np.zeros((3, n))
    u[0] = u_in
    for k in range(3):
        u[k] += 1e-3 * u_in * uniform_at(SPHERE_SEED, level, coords, k)
    return np.ones(n), u


# ------------------------------------------------------------------ 2D flow past a NACA0012 airfoil
# Level boxes as multiples of the chord C around the leading edge (x) and the chord line (y),
# finest level first; the domain is [-15C, 15C]^2 and the coarsest level fills the rest.
NACA_BOXES = [((-0.1, 1.1), (-0.15, 0.15)), ((-0.5, 2.0), (-0.5, 0.5)), ((-2.0, 5.0), (-2.0, 2.0)),
              ((-6.0, 12.0), (-6.0, 6.0))]
NACA_SEED = 1504


# Reduced form for parity runs at small chords: the finest box is wide enough that the airfoil
# stays more than the reach of the 37- and 21-velocity lattices (3 cells) from its fine ghosts.
NACA_BOXES_SMALL = [((-0.25, 1.25), (-0.3, 0.3)), ((-0.75, 2.0), (-0.75, 0.75))]


def naca_spec(chord: int, mach: float, T0: float, gamma: float = 1.4, n_levels: int = 5,
              supersonic: bool = True, half_domain: float = 15.0, level_boxes=None) -> GridSpec:
    """Multi-level box around a NACA0012 at zero incidence, chord ``chord`` finest cells.

    The domain is [-h C, h C]^2 around the leading edge (h = ``half_domain``), which sits at the
    domain centre.  Inflow at x-: every macroscopic field imposed (supersonic inlet) or density
    extrapolated (subsonic); Neumann on the other faces.  ``level_boxes`` (default NACA_BOXES)
    gives the refined boxes in chords, finest level first; box edges are rounded outwards to
    whole cells of the next coarser level."""
    ext = int(round(2 * half_domain * chord))
    cx, cy = ext // 2, ext // 2
    boxes = []
    for lev, ((x0, x1), (y0, y1)) in enumerate((level_boxes or NACA_BOXES)[:n_levels - 1]):
        a = 2 ** (lev + 1)
        lo = (int(np.floor((cx + x0 * chord) / a)) * a, int(np.floor((cy + y0 * chord) / a)) * a)
        hi = (int(np.ceil((cx + x1 * chord) / a)) * a, int(np.ceil((cy + y1 * chord) / a)) * a)
        boxes.append((lev, lo, hi))
    u_in = mach * np.sqrt(gamma * T0)
    inflow = ("dirichlet", 1.0, (u_in, 0.0, 0.0), T0) if supersonic else ("dirichlet_rho", 1.0, (u_in, 0.0, 0.0), T0)
    faces = {"x-": inflow, "x+": ("neumann",), "y-": ("neumann",), "y+": ("neumann",)}
    return GridSpec(2, (ext, ext), n_levels, boxes[::-1], (False, False), faces,
                    [{"kind": "naca", "chord": float(chord), "x0": float(cx), "y0": float(cy), "thickness": 0.12}])


def naca_fields(level, coords: np.ndarray, mach: float, T0: float, gamma: float = 1.4):
    """Uniform free stream rho = 1, u = Ma sqrt(gamma T0) (1, 0) with a 1e-3 relative
    perturbation per cell (splitmix64, seed 1504), T = T0."""
    coords = np.asarray(coords)
    n = coords.shape[0]
    u_in = mach * np.sqrt(gamma * T0)
    u = np.zeros((2, n))
    u[0] = u_in * (1.0 + 1e-3 * uniform_at(NACA_SEED, level, coords, 0))
    u[1] = 1e-3 * u_in * uniform_at(NACA_SEED, level, coords, 1)
    return np.ones(n), u, np.full(n, T0)


# ------------------------------------------------------------------ batch of uneven 2D cases
def _place_boxes(rng, parents, n_boxes, unit, margin, frac=(0.3, 0.55), min_cells=32):
    """Up to n_boxes disjoint boxes, each inside one of the parent boxes (lo, hi) with
    ``margin`` parent cells of clearance from the parent's edges and from each other; edges on
    multiples of ``unit`` finest units (8 parent cells)."""
    out = []
    for _ in range(n_boxes):
        for _attempt in range(20):
            plo, phi = parents[rng.integers(len(parents))]
            lo, hi = [], []
            ok = True
            for d in range(2):
                span = phi[d] - plo[d]
                size = int(rng.uniform(*frac) * span) // unit * unit
                room = span - size - 2 * margin
                if size < min_cells * unit // 8 or room < 0:
                    ok = False
                    break
                start = plo[d] + margin + int(rng.integers(0, room // unit + 1)) * unit
                lo.append(start)
                hi.append(start + size)
            if not ok:
                continue
            clash = any(all(lo[d] < b_hi[d] + margin and b_lo[d] < hi[d] + margin for d in range(2))
                        for b_lo, b_hi in out)
            if not clash:
                out.append((tuple(lo), tuple(hi)))
                break
    return out


def batch_cases(seed: int = 48, n: int = 48):
    """Uneven 2D cases for batched stepping (PCG64 stream ``seed``): coarse sides 2^U{6..10},
    2-4 levels, 1-3 refined boxes per level nested in the next coarser level's boxes, half
    D2Q9 recursive-regularized Taylor-Green, half D2Q37 polynomial-DDF Sod tubes along x.

    Returns dicts {name, lattice, model, spec, fields(level, coords) -> (rho, u[, T]), params}."""
    rng = np.random.default_rng(seed)
    cases = []
    for k in range(n):
        L = int(rng.integers(2, 5))
        s = 2 ** (L - 1)
        tg = (k % 2 == 0)
        if tg:
            cx = cy = 2 ** int(rng.integers(6, 11))
        else:
            cx = 2 ** int(rng.integers(7, 11))
            cy = 2 ** int(rng.integers(6, min(int(np.log2(cx)), 9) + 1))
        ext = (cx * s, cy * s)
        boxes = []
        parents = [((0, 0), ext)]
        for lev in range(L - 2, -1, -1):
            unit = 8 * 2 ** (lev + 1)                  # 8 cells of the parent level
            margin = 16 * 2 ** (lev + 1)
            placed = _place_boxes(rng, parents, int(rng.integers(1, 4)), unit, margin)
            if not placed:
                break
            boxes += [(lev, lo, hi) for lo, hi in placed]
            parents = placed
        levels = L if boxes else 1
        if levels < L:                                 # drop the empty finer levels
            shift = L - levels
            ext = (ext[0] >> shift, ext[1] >> shift)
            boxes = [(lev - shift, tuple(v >> shift for v in lo), tuple(v >> shift for v in hi)) for lev, lo, hi in boxes]
        if tg:
            spec = GridSpec(2, ext, levels, boxes, (True, True))
            u0, nc = 0.05, cx

            def fields(level, coords, nc=nc, levels=levels, u0=u0):
                c = cell_centres(coords, level)
                return taylor_green_fields(c, nc, levels, u0, 1.0 / 3.0)
            cases.append({"name": f"tg{k}", "lattice": "D2Q9", "model": "rr", "spec": spec, "fields": fields,
                          "params": {"nu0": 0.01 * 2 ** (levels - 1)}})
        else:
            spec = GridSpec(2, ext, levels, boxes, (False, True), {"x-": ("neumann",), "x+": ("neumann",)})
            T0 = 0.7

            def fields(level, coords, nx=ext[0], T0=T0):
                return sod_fields(cell_centres(coords, level), nx, T0)
            cases.append({"name": f"sod{k}", "lattice": "D2Q37", "model": "poly_ddf", "spec": spec, "fields": fields,
                          "params": {"nu0": 0.0, "T0": T0, "sensor_A": 1.5}})
    return cases
