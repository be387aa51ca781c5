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
