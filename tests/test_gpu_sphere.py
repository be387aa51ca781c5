"""The benchmark workload (D3Q27 RR flow past a sphere, 4 levels) against the oracle.

* the reduced copy (extents / 4, sphere D = 16, same level structure) for 2 coarse steps,
  FP64 (relative L2 <= 1e-12) and FP32 (<= 1e-5);
* the full 1024x512x512 workload in the benchmark's launch configuration (FP32, its block shape
  and kernel variant): after one fine iteration, rho and u at 2000 sampled interior level-0 cells
  against the oracle's local computation (equilibrium of the seeded fields, RR collision,
  streaming from the 27 neighbours).
"""
from functools import lru_cache

import numpy as np
import pytest

from oracle import hermite as hm
from oracle import lattices as L
from paper_2504_04465_b300 import inputs as I

from . import harness as H

pytestmark = pytest.mark.gpu


def _fields(level, coords, c):
    return I.sphere_fields(level, coords)


@lru_cache(maxsize=None)
def reduced_oracle():
    return H.run_oracle(I.sphere_spec(4), "D3Q27", "rr", _fields, 16, nu0=I.sphere_nu0(4))


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_reduced_sphere_four_levels(storage, tol):
    sol = reduced_oracle()
    ctx = H.make_gpu(I.sphere_spec(4), "D3Q27", "rr", storage, _fields, nu0=I.sphere_nu0(4))
    ctx.step(2)
    err = H.compare_moments(sol, ctx)
    print("reduced sphere", storage, err)
    assert err["rho"] < tol and err["u"] < tol, err


def test_full_sphere_sampled_first_iteration():
    import bench
    from paper_2504_04465_b300 import lbmtree as lt
    spec = I.sphere_spec(1)
    block = bench.DEFAULT_BLOCK["f32"]
    ctx = lt.Context(3, device=0)
    ctx.configure(spec, "D3Q27", "rr", "f32", block=block, nu0=I.sphere_nu0(1))
    ctx.set_variant(bench.DEFAULT_VARIANT["f32"])
    ctx.use_graph(True)
    rho0, u0 = bench.host_fields(ctx)
    ctx.init_fields(rho0, u0)
    ctx.step_fine(1)
    rho_g, u_g, _ = ctx.moments()
    lv, xyz, ty = ctx.cells()
    # interior level-0 cells: 4 cells inside the level-0 box, 4 cells outside the sphere
    lo = np.array([160, 128, 128]) + 4
    hi = np.array([672, 384, 384]) - 4
    m = (lv == 0) & np.all(xyz >= lo, axis=1) & np.all(xyz < hi, axis=1)
    r = np.sqrt(((xyz + 0.5 - np.array([256.0, 256.0, 256.0])) ** 2).sum(axis=1))
    m &= r > 32.0 + 4
    idx = np.nonzero(m)[0]
    rng = np.random.default_rng(3900)
    pick = rng.choice(idx, size=2000, replace=False)
    lat = L.D3Q27
    tau = I.sphere_nu0(1) / lat.cs2 + 0.5
    x = xyz[pick]
    f_new = np.zeros((lat.Q, pick.size))
    for q in range(lat.Q):
        y = x - lat.xi[q][None, :]
        rho, u = I.sphere_fields(0, y)
        feq = hm.feq_athermal(lat, rho, u)
        fs = hm.collide_rr(lat, feq, tau)
        f_new[q] = fs[q]
    rho_o = f_new.sum(axis=0)
    u_o = (lat.xi.T.astype(float) @ f_new) / rho_o
    err_rho = np.abs(rho_g[pick] - rho_o).max()
    err_u = np.abs(u_g[:, pick] - u_o).max() / np.abs(u_o).max()
    print("full sphere sampled", err_rho, err_u)
    assert err_rho < 1e-6 and err_u < 1e-5
