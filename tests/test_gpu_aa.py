"""AA-pattern in-place streaming (GPU required): one population buffer, even iterations on each
cell's own slots, odd iterations gathering from and writing back to the neighbours.  The same
collisions run on the same values as with two buffers, so every readout is bitwise that of the
two-buffer path (FP64 and FP32, after odd and even iteration counts, plain launches and CUDA
graphs), with half the population memory; the FP64 results also match the oracle to 1e-12."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2504_04465_b300 import inputs as I
from tests import harness as H

pytestmark = pytest.mark.gpu


def rest(level, coords, c):
    return np.ones(c.shape[0]), np.zeros((c.shape[1], c.shape[0]))


def fields3(level, coords, c):
    rho = 1.0 + 0.02 * I.uniform_at(61, level, coords, 0)
    u = 0.04 * np.stack([I.uniform_at(62, level, coords, k) for k in range(3)])
    return rho, u


SPHERE_BOX = I.GridSpec(3, (64, 32, 32), 1, [], (True, True, True),
                        solids=[{"kind": "sphere", "center": (32.0, 16.0, 16.0), "radius": 6.0}])
CLOSED37 = I.GridSpec(2, (128, 32), 1, [], (False, True), {f: ("wall", 1.0, (0.0, 0.0, 0.0)) for f in ("x-", "x+")})
INLET9 = I.GridSpec(2, (128, 64), 1, [], (False, True),
                    {"x-": ("dirichlet", 1.0, (0.05, 0.0, 0.0)), "x+": ("dirichlet", 1.0, (0.05, 0.0, 0.0))},
                    [{"kind": "sphere", "center": (40.0, 32.0), "radius": 6.0}])


def _sod37(level, coords, c):
    from paper_2504_04465_b300 import lbmtree as lt
    return I.sod_fields(c, 128, lt.lattice_cs2("D2Q37"))


CASES = [
    ("tg_q9_rr", I.taylor_green_spec(256, 0, 0, 1), "D2Q9", "rr", H.tg_fields(256, 1, seed=7, amp=0.01), dict(nu0=0.01)),
    ("cavity_q9_bgk", I.cavity_spec(64, 0.1), "D2Q9", "bgk", rest, dict(nu0=0.02)),
    ("inlet_sphere_q9_rr", INLET9, "D2Q9", "rr", rest, dict(nu0=0.02)),
    ("sphere_q27_rr", SPHERE_BOX, "D3Q27", "rr", fields3, dict(nu0=0.02)),
    ("cavity_q27_bgk", I.cavity_spec(32, 0.05, dim=3), "D3Q27", "bgk", rest, dict(nu0=0.02)),
    ("closed_q37_poly", CLOSED37, "D2Q37", "poly_ddf", _sod37, dict(nu0=0.0, sensor_A=1.5)),
]


def _read(ctx, comp):
    rho, u, T = ctx.moments()
    out = [rho, u, ctx.populations("f")]
    if comp:
        out += [T, ctx.populations("g")]
    return out


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("name,spec,lat,model,fields,kw", CASES, ids=[c[0] for c in CASES])
def test_aa_bitwise_equals_two_buffers(name, spec, lat, model, fields, kw, storage):
    comp = model.endswith("ddf")
    ab = H.make_gpu(spec, lat, model, storage, fields, **kw)
    aa = H.make_gpu(spec, lat, model, storage, fields, streaming="aa", **kw)
    for n in (1, 6):                     # after 1 and 7 iterations (layout L0), then 8 (L1)
        ab.step_fine(n)
        aa.step_fine(n)
        for x, y in zip(_read(ab, comp), _read(aa, comp)):
            assert np.array_equal(x, y), name
    aa.use_graph(True)
    ab.step_fine(1)
    aa.step_fine(1)
    ab.step_fine(8)
    aa.step_fine(8)                      # four captured two-iteration spans
    aa.sync()
    for x, y in zip(_read(ab, comp), _read(aa, comp)):
        assert np.array_equal(x, y), name
    assert np.array_equal(ab.conserved(), aa.conserved())
    s_ab, s_aa = ab.stats(), aa.stats()
    Q = ab.velocities().shape[0]
    es = 8 if storage == "f64" else 4
    nslots = s_ab.n_blocks[0] * np.prod(s_ab.block) + np.prod(s_ab.block)
    saved = Q * nslots * es * (2 if comp else 1)
    assert s_ab.device_bytes - s_aa.device_bytes >= 0.99 * saved
    ab.close()
    aa.close()


@pytest.mark.parametrize("name,spec,lat,model,fields,kw", CASES[1:4], ids=[c[0] for c in CASES[1:4]])
def test_aa_matches_oracle(name, spec, lat, model, fields, kw):
    n = 9
    sol = H.run_oracle(spec, lat, model, fields, n, **kw)
    ctx = H.make_gpu(spec, lat, model, "f64", fields, streaming="aa", **kw)
    ctx.step_fine(n)
    ctx.sync()
    err = H.compare_moments(sol, ctx)
    print(name, "aa", err)
    assert err["rho"] < 1e-12 and err["u"] < 1e-12, err
    assert H.compare_populations(sol, ctx) < 1e-12
    ctx.close()


def test_aa_full_size_box_bitwise():
    """At the aa form's size (512 x 256 x 256 D3Q27 RR, FP32, 33.6 M cells): AA and two-buffer
    streaming give the same moments and totals bit for bit after 3 and 4 iterations."""
    spec = I.GridSpec(3, (512, 256, 256), 1, [], (True, True, True))

    def fields(level, coords, c):
        rho = 1.0 + 1e-3 * I.uniform_at(71, level, coords, 0)
        u = 0.02 + 1e-3 * np.stack([I.uniform_at(72 + k, level, coords, 0) for k in range(3)])
        return rho, u
    ab = H.make_gpu(spec, "D3Q27", "rr", "f32", fields, nu0=0.01)
    aa = H.make_gpu(spec, "D3Q27", "rr", "f32", fields, nu0=0.01, streaming="aa")
    for n in (3, 1):
        ab.step_fine(n)
        aa.step_fine(n)
        ra, rb = ab.moments(), aa.moments()
        assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
        assert np.array_equal(ab.conserved(), aa.conserved())
    ab.close()
    aa.close()
