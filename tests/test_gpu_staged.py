"""The binary16 interior kernel of the D3Q27 regularized model (the default in binary16
deviation storage: pull staged in shared memory, two cells per thread, the collision in packed
FP32 pairs on the stored relative deviations) against the kernel that gathers straight from global
memory and collides through the general weakly compressible path (the variants with codes >= 100).

Both compute the same regularized collision in FP32 and round it to binary16; they differ only in
the order of FP32 operations (about 1e-8 of the populations), so after one iteration the
stored deviations h = f / (w rho_ref) - 1 agree to one binary16 unit in the last place, and rarely
differ at all.  Over ten coarse steps the moments of the two paths stay within the binary16 error, and
the staged path keeps the bound stated against the FP64 oracle.  Cases: the two-level sphere with
a Dirichlet inlet and a Neumann outlet (simple, streaming and general blocks), the four-level
reduced benchmark sphere (fine ghosts in streaming blocks), and the 8x8x2 block shape.
"""
import numpy as np
import pytest

from paper_2504_04465_b300 import inputs as I

from . import harness as H
from .test_gpu_parity import D3_SPEC, d3_fields, d3_oracle

pytestmark = pytest.mark.gpu


def _weights(ctx):
    """D3Q27 weights in the library's velocity order: products of 2/3 (xi_a = 0) and 1/6."""
    xi = ctx.velocities()
    return np.prod(np.where(xi == 0, 2.0 / 3.0, 1.0 / 6.0), axis=1)


def _ctx(spec, fields, nu0, code, block=None):
    ctx = H.make_gpu(spec, "D3Q27", "rr", "f16dev", fields, block=block, nu0=nu0)
    ctx.set_variant(ctx.variants().index(code))
    return ctx


def _rel_dev(ctx):
    """Stored relative deviations h = f / (w rho_ref) - 1 (rho_ref = 1)."""
    f = ctx.populations("f")
    return f / _weights(ctx)[:, None] - 1.0


def _ulp16(x):
    """Binary16 spacing at |x| (normal range; 2^-24 below it)."""
    a = np.maximum(np.abs(x), 2.0 ** -14)
    return np.where(np.abs(x) < 2.0 ** -14, 2.0 ** -24, 2.0 ** (np.floor(np.log2(a)) - 10))


def _agreement(spec, fields, nu0, code, n_fine, block=None):
    """Stored deviations of the staged and the direct path after n_fine fine iterations from the
    same state.  One iteration: at most one binary16 ulp apart.  More: a one-ulp difference in an
    input moves a collided output by about the input's ulp, so four ulps of max(|h|, 1/64)."""
    a = _ctx(spec, fields, nu0, code, block)
    b = _ctx(spec, fields, nu0, 100 + code, block)
    a.step_fine(n_fine)
    b.step_fine(n_fine)
    ha, hb = _rel_dev(a), _rel_dev(b)
    assert np.isfinite(ha).all() and np.isfinite(hb).all()
    d = np.abs(ha - hb)
    mag = np.maximum(np.abs(ha), np.abs(hb))
    if n_fine == 1:
        tol = _ulp16(mag) * 1.001 + 1e-7
    else:
        tol = 4.0 * _ulp16(np.maximum(mag, 1.0 / 64.0))
    frac = float(np.mean(d > 1e-7))
    print("staged vs direct after", n_fine, "iterations: max |dh| / tol", float((d / tol).max()),
          "fraction differing", frac)
    assert (d <= tol).all()
    assert frac < 0.01
    return a


def test_variant_codes():
    ctx = H.make_gpu(D3_SPEC, "D3Q27", "rr", "f16dev", d3_fields, nu0=0.01)
    assert np.isclose(_weights(ctx).sum(), 1.0)
    codes = ctx.variants()
    staged = [c for c in codes if c < 100]
    direct = [c for c in codes if c >= 100]
    assert len(staged) == len(direct) == 4 and [c - 100 for c in direct] == staged
    ctx32 = H.make_gpu(D3_SPEC, "D3Q27", "rr", "f32", d3_fields, nu0=0.01)
    assert all(c < 100 for c in ctx32.variants())


@pytest.mark.parametrize("code", [0, 86, 88])
@pytest.mark.parametrize("n_fine", [1, 4])
def test_two_level_sphere(code, n_fine):
    _agreement(D3_SPEC, d3_fields, 0.01, code, n_fine)


def test_reduced_benchmark_sphere_fine_ghosts():
    # fine iterations 1-4 of the four-level grid: every level's fine ghosts both receive
    # explosions and stream through the interior kernel
    def fields(level, coords, c):
        return I.sphere_fields(level, coords)
    _agreement(I.sphere_spec(4), fields, I.sphere_nu0(4), 86, 4)


def test_block_8x8x2():
    _agreement(D3_SPEC, d3_fields, 0.01, 0, 1, block=(8, 8, 2))


def test_ten_coarse_steps_within_binary16_error():
    sol = d3_oracle()
    a = _ctx(D3_SPEC, d3_fields, 0.01, 86)
    b = _ctx(D3_SPEC, d3_fields, 0.01, 186)
    a.step(10)
    b.step(10)
    ea, eb = H.compare_moments(sol, a), H.compare_moments(sol, b)
    print("staged", ea, "direct", eb)
    assert ea["rho"] < 3e-2 and ea["u"] < 3e-2, ea
    assert ea["rho"] < 1.5 * eb["rho"] + 1e-6 and ea["u"] < 1.5 * eb["u"] + 1e-5
    ra, ua, _ = a.moments()
    rb, ub, _ = b.moments()
    assert H.rel_l2(ra, rb) < 1e-4 and H.rel_l2(ua, ub) < 2e-3


# Neumann faces across y: their boundary cells' partners sit in other threads of the block, so
# the staged kernel hands the partner's result over through a block barrier
D3_YN_SPEC = I.GridSpec(3, (64, 32, 32), 2, [(0, (16, 8, 8), (48, 24, 24))], (False, False, True),
                        {"x-": ("dirichlet_rho", 1.0, (0.04, 0.0, 0.0)), "x+": ("neumann",),
                         "y-": ("neumann",), "y+": ("neumann",)},
                        [{"kind": "sphere", "center": (32.0, 16.0, 16.0), "radius": 4.0}])


@pytest.mark.parametrize("n_fine", [1, 4])
def test_neumann_faces_across_y(n_fine):
    _agreement(D3_YN_SPEC, d3_fields, 0.01, 86, n_fine)


def test_neumann_faces_across_y_against_oracle():
    sol = H.run_oracle(D3_YN_SPEC, "D3Q27", "rr", d3_fields, 2 * 6, nu0=0.01)
    ctx = _ctx(D3_YN_SPEC, d3_fields, 0.01, 86)
    ctx.step(6)
    err = H.compare_moments(sol, ctx)
    assert err["rho"] < 3e-2 and err["u"] < 3e-2, err
    # a Neumann boundary cell of the y- face (coarse level, away from the x faces) holds its
    # partner's state exactly: the same binary16 bits
    lv, xyz, ty = ctx.cells()
    f = ctx.populations("f")
    m = (lv == 1) & (xyz[:, 1] == 0) & (xyz[:, 0] >= 4) & (xyz[:, 0] < 28)
    key = {(int(a), int(b), int(c), int(d)): i for i, (a, (b, c, d)) in enumerate(zip(lv, xyz))}
    idx = np.nonzero(m)[0]
    assert idx.size > 0
    for i in idx:
        j = key[(1, int(xyz[i, 0]), 1, int(xyz[i, 2]))]
        assert np.array_equal(f[:, i], f[:, j])
