"""C-ABI checks that need no GPU: the library loads, exports every declared entry point, rejects
bad calls with the documented codes, and its host grid builder reproduces the oracle's cell sets
(host-only contexts, device < 0, run no kernel)."""
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import grid as G
from oracle import lattices as L
from paper_2504_04465_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbmtree.h")


@pytest.fixture(scope="module")
def lt():
    from paper_2504_04465_b300.build import build
    build()
    from paper_2504_04465_b300 import lbmtree
    return lbmtree


def declared_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(lbm_\w+)\s*\(", txt, flags=re.M)))


def test_every_declared_symbol_is_exported(lt):
    names = declared_functions()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", lt.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(lbm_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert set(names) <= set(lt.EXPORTED)


def test_build_targets_sm103a():
    from paper_2504_04465_b300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_bad_arguments(lt):
    with pytest.raises(lt.LbmError) as e:
        lt.Context(4, device=-1)
    assert e.value.code == -1
    c = lt.Context(2, device=-1)
    with pytest.raises(lt.LbmError):
        c.set_lattice("D3Q27")                       # dimension mismatch
    c.set_lattice("D2Q9")
    with pytest.raises(lt.LbmError) as e:
        c.build_grid((64, 64), 1)                    # collision model not set
    assert e.value.code == -2
    c.set_collision("rr", nu0=0.01)
    with pytest.raises(lt.LbmError) as e:
        c.step(1)                                    # nothing built
    assert e.value.code == -2
    with pytest.raises(lt.LbmError) as e:            # misaligned box
        c.build_grid((64, 64), 2, [(0, (15, 16), (48, 48))])
    assert e.value.code == -5
    c2 = lt.Context(2, device=-1)
    c2.set_lattice("D2Q9")
    c2.set_collision("poly_ddf")
    with pytest.raises(lt.LbmError) as e:
        c2.build_grid((64, 64), 1)
    assert e.value.code == -10


def _compare(lt, spec, latname, model, block=None):
    g = G.build(spec, L.LATTICES[latname])
    c = lt.Context(spec.dim, device=-1)
    c.configure(spec, latname, model, block=block)
    lv, xyz, ty = c.cells()
    for i, olv in enumerate(g.levels):
        m = lv == i
        got = {tuple(int(a) for a in x[: spec.dim]): int(t) for x, t in zip(xyz[m], ty[m])}
        exp = {tuple(int(v) for v in x): int(t) for x, t in zip(olv.coords, olv.ctype)}
        assert got == exp, i
    assert c.stats().n_eq == pytest.approx(g.n_eq())
    return c


SPECS = [
    ("tg2", lambda: I.taylor_green_spec(64, 16, 48, 2), "D2Q9", "rr", None),
    ("tg2_32x8", lambda: I.taylor_green_spec(64, 16, 48, 2), "D2Q9", "bgk", (32, 8, 1)),
    ("three_levels", lambda: I.GridSpec(2, (128, 128), 3, [(1, (32, 32), (96, 96)), (0, (48, 48), (80, 80))], (True, True)), "D2Q9", "bgk", None),
    ("reach3_q37", lambda: I.GridSpec(2, (96, 64), 2, [(0, (32, 16), (64, 48))], (True, True)), "D2Q37", "poly_ddf", None),
    ("reach3_q21", lambda: I.GridSpec(2, (96, 64), 2, [(0, (32, 16), (64, 48))], (True, True)), "D2Q21", "num_ddf", None),
    ("riemann12_diag_q21", lambda: I.riemann12_spec(16, "diag"), "D2Q21", "num_ddf", None),
    ("riemann12_optim_q37", lambda: I.riemann12_spec(16, "optim"), "D2Q37", "num_ddf", None),
    ("reach2_q13", lambda: I.GridSpec(2, (96, 64), 2, [(0, (32, 16), (64, 48))], (True, True)), "D2Q13", "rr", None),
    ("reach2_q13_sod", lambda: I.sod_spec(256, 32, 2, (64, 192)), "D2Q13", "num_ddf", None),
    ("reach2_q13_naca", lambda: I.naca_spec(64, 0.8, 0.35, n_levels=3, supersonic=False, half_domain=3.0,
                                            level_boxes=I.NACA_BOXES_SMALL), "D2Q13", "num_ddf", None),
    ("sod_band", lambda: I.sod_spec(256, 32, 2, (64, 192)), "D2Q37", "poly_ddf", None),
    ("solid", lambda: I.GridSpec(2, (64, 64), 2, [(0, (16, 16), (48, 48))], (True, True),
                                 solids=[{"kind": "sphere", "center": (32.0, 32.0), "radius": 5.0}]), "D2Q9", "rr", None),
    ("channel_ragged", lambda: I.GridSpec(2, (200, 128), 3, [(1, (40, 32), (160, 96)), (0, (64, 48), (128, 80))], (False, True),
                                          {"x-": ("dirichlet_rho", 1.0, (0.05, 0.0, 0.0)), "x+": ("neumann",)},
                                          [{"kind": "sphere", "center": (88.0, 64.0), "radius": 6.0}]), "D2Q9", "rr", None),
    ("naca", lambda: I.GridSpec(2, (256, 128), 2, [(0, (64, 32), (192, 96))], (False, False),
                                {f: ("neumann",) for f in ("x-", "x+", "y-", "y+")},
                                [{"kind": "naca", "chord": 80.0, "x0": 88.0, "y0": 64.0}]), "D2Q21", "num_ddf", None),
    ("d3q27_sphere", lambda: I.GridSpec(3, (64, 32, 32), 2, [(0, (16, 8, 8), (48, 24, 24))], (False, True, True),
                                        {"x-": ("dirichlet_rho", 1.0, (0.04, 0.0, 0.0)), "x+": ("neumann",)},
                                        [{"kind": "sphere", "center": (32.0, 16.0, 16.0), "radius": 4.0}]), "D3Q27", "rr", None),
]


@pytest.mark.parametrize("name,mk,latname,model,block", SPECS, ids=[s[0] for s in SPECS])
def test_host_builder_matches_oracle(lt, name, mk, latname, model, block):
    _compare(lt, mk(), latname, model, block)


def test_velocity_sets_match_oracle(lt):
    for latname, dim, model in (("D2Q9", 2, "rr"), ("D2Q13", 2, "rr"), ("D2Q21", 2, "num_ddf"), ("D2Q37", 2, "poly_ddf"),
                                ("D3Q27", 3, "rr")):
        c = lt.Context(dim, device=-1)
        c.set_lattice(latname)
        c.set_collision(model)
        ext = (32, 32) if dim == 2 else (8, 8, 8)
        c.build_grid(ext, 1)
        xi = c.velocities()[:, :dim]
        assert {tuple(int(a) for a in v) for v in xi} == {tuple(int(a) for a in v) for v in L.LATTICES[latname].xi}
        assert np.array_equal(xi[::-1], -xi)          # opposite of q is Q-1-q


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("fp32", [False, True])
def test_numerical_equilibrium_lattices(lt, storage, fp32):
    """The numerical equilibrium is built on D2Q13, D2Q21 and D2Q37 (Appendix A.2), for either Newton
    precision (D2Q13: the FP32 solve with FP32 populations only); D2Q9 refuses it."""
    for latname in ("D2Q13", "D2Q21", "D2Q37"):
        if latname == "D2Q13" and fp32 and storage != "f32":
            continue
        c = lt.Context(2, device=-1)
        c.configure(I.GridSpec(2, (32, 32), 1, [], (True, True)), latname, "num_ddf", storage, T0=0.9,
                    newton_fp32=fp32)
        assert c.n_cells() == 32 * 32
    c = lt.Context(2, device=-1)
    with pytest.raises(lt.LbmError) as e:
        c.configure(I.GridSpec(2, (32, 32), 1, [], (True, True)), "D2Q9", "num_ddf", storage, T0=0.9,
                    newton_fp32=fp32)
    assert lt.ERR[e.value.code] == "UNSUPPORTED"


def test_batch_needs_initialised_device_contexts(lt):
    ctx = lt.Context(2, device=-1)
    ctx.configure(I.taylor_green_spec(32, 8, 24, 2), "D2Q9", "rr", "f64", nu0=0.02)
    with pytest.raises(lt.LbmError) as e:
        lt.Batch([ctx])
    assert lt.ERR[e.value.code] == "STATE"
    with pytest.raises(lt.LbmError):
        lt.Batch([])


def test_batch_case_recipe_builds(lt):
    cases = I.batch_cases()
    assert len(cases) == 48
    assert sum(c["lattice"] == "D2Q9" for c in cases) == 24
    total = 0
    levels = set()
    for c in cases:
        ctx = lt.Context(2, device=-1)
        ctx.configure(c["spec"], c["lattice"], c["model"], "f32", **c["params"])
        s = ctx.stats()
        total += int(sum(s.n_cells[:s.n_levels]))
        levels.add(s.n_levels)
        ctx.close()
    assert 20e6 <= total <= 30e6, total
    assert levels == {2, 3, 4}


def test_lattice_info_matches_the_oracle_lattices(lt):
    for name in ("D2Q9", "D2Q13", "D2Q21", "D2Q37", "D3Q27"):
        info = lt.lattice_info(name)
        ref = L.LATTICES[name]
        assert info["Q"] == ref.Q and info["D"] == ref.D
        assert abs(info["cs2"] - ref.cs2) < 1e-14
    with pytest.raises(lt.LbmError):
        lt._check(lt._lib.lbm_lattice_info(15, None, None, None, None), "lbm_lattice_info")


def test_checkpoint_calls_check_their_arguments(lt, tmp_path):
    ctx = lt.Context(2, device=-1)
    ctx.configure(I.taylor_green_spec(32, 8, 24, 2), "D2Q9", "rr", "f64", nu0=0.02)
    with pytest.raises(lt.LbmError):
        ctx.save(str(tmp_path / "a.ckpt"))          # host-only context: nothing to save
    with pytest.raises(lt.LbmError):
        ctx.load(str(tmp_path / "missing.ckpt"))


def test_collision_variant_arguments(lt):
    c = lt.Context(2, device=-1)
    c.set_lattice("D2Q9")
    with pytest.raises(lt.LbmError) as e:
        c.set_collision("trt", nu0=0.0)                  # TRT needs a viscosity
    assert e.value.code == -1
    with pytest.raises(lt.LbmError):
        c.set_collision("bgk", nu0=0.01, trace_eq=True)  # trace equilibration is an RR option
    with pytest.raises(lt.LbmError):
        c.set_sponge((0, 0, 0), 10.0, 5.0, 0.1)          # r1 <= r0
    with pytest.raises(lt.LbmError):
        c.set_sponge((0, 0, 0), 5.0, 10.0, 1.5)          # sigma_max > 1
    c.set_collision("trt", nu0=0.01)
    c.set_precision("f16dev")
    with pytest.raises(lt.LbmError) as e:
        c.build_grid((64, 64), 1)                        # TRT: FP64 and FP32 storage only
    assert e.value.code == -10
    c2 = lt.Context(2, device=-1)
    c2.set_lattice("D2Q21")
    c2.set_collision("trt", nu0=0.01)
    with pytest.raises(lt.LbmError) as e:
        c2.build_grid((64, 64), 1)                       # TRT built on D2Q9 and D3Q27
    assert e.value.code == -10
    c3 = lt.Context(2, device=-1)
    c3.set_lattice("D2Q37")
    c3.set_collision("poly_ddf", nu0=0.01)
    with pytest.raises(lt.LbmError) as e:
        c3.set_sponge((0, 0, 0), 5.0, 10.0, 0.1)         # weakly compressible models only
    assert e.value.code == -10
    c4 = lt.Context(2, device=-1)
    c4.set_lattice("D2Q9")
    c4.set_collision("rr", nu0=0.01, trace_eq=True)
    c4.set_sponge((32, 32, 0), 5.0, 10.0, 0.1)
    c4.build_grid((64, 64), 1)


WALL_SPECS = [
    ("cavity_q9", lambda: I.cavity_spec(64, 0.1, 2, (16, 48)), "D2Q9", "rr"),
    ("cavity_q27", lambda: I.cavity_spec(32, 0.05, 2, (8, 24), dim=3), "D3Q27", "rr"),
    ("couette_q9", lambda: I.couette_spec(32, 16, 0.05), "D2Q9", "bgk"),
    ("closed_q37", lambda: I.GridSpec(2, (128, 32), 1, [], (False, True),
                                      {f: ("wall", 1.0, (0.0, 0.0, 0.0)) for f in ("x-", "x+")}), "D2Q37", "poly_ddf"),
]


@pytest.mark.parametrize("name,mk,latname,model", WALL_SPECS, ids=[s[0] for s in WALL_SPECS])
def test_wall_grids_match_oracle(lt, name, mk, latname, model):
    _compare(lt, mk(), latname, model)


def test_wall_arguments(lt):
    c = lt.Context(2, device=-1)
    c.set_lattice("D2Q9")
    c.set_collision("rr", nu0=0.01)
    with pytest.raises(lt.LbmError):
        c.configure(I.cavity_spec(64, 0.1, 2, (0, 32)), "D2Q9", "rr")      # ghosts next to a wall
    c2 = lt.Context(2, device=-1)
    with pytest.raises(lt.LbmError) as e:                                   # moving wall, compressible
        c2.configure(I.GridSpec(2, (128, 32), 1, [], (False, True),
                                {"x-": ("wall", 1.0, (0.0, 0.1, 0.0)), "x+": ("wall",)}), "D2Q37", "poly_ddf")
    assert e.value.code == -10


def test_aa_streaming_arguments(lt):
    from tests.test_gpu_aa import CASES
    for name, spec, latname, model, _, kw in CASES:           # every AA case builds
        c = lt.Context(spec.dim, device=-1)
        c.configure(spec, latname, model, "f32", streaming="aa", **{k: v for k, v in kw.items()})
    bad = [
        (I.taylor_green_spec(64, 16, 48, 2), "D2Q9", "rr", "f64"),                      # two levels
        (I.sod_spec(256, 32), "D2Q37", "poly_ddf", "f64"),                              # Neumann faces
        (I.GridSpec(2, (64, 64), 1, [], (True, True)), "D2Q21", "num_ddf", "f64"),     # not compiled
        (I.GridSpec(2, (64, 64), 1, [], (True, True)), "D2Q9", "trt", "f64"),          # not compiled
    ]
    for spec, latname, model, st in bad:
        c = lt.Context(2, device=-1)
        with pytest.raises(lt.LbmError) as e:
            c.configure(spec, latname, model, st, streaming="aa", nu0=0.02)
        assert e.value.code == -10, (latname, model)
    c = lt.Context(2, device=-1)
    with pytest.raises(lt.LbmError):
        lt._check(lt._lib.lbm_set_streaming(c._h, 7), "lbm_set_streaming")    # unknown mode


def test_neumann_end_blocks_are_interior_blocks():
    """Blocks whose only boundary cells are Neumann cells with their partner in the block run in
    the interior kernel (list entries with the streaming bit): a Sod tube with Neumann ends has
    no general block; imposing the density at one end makes that end's blocks general."""
    from paper_2504_04465_b300 import lbmtree as lt
    ny = 32
    c = lt.Context(2, device=-1)
    c.configure(I.sod_spec(256, ny), "D2Q37", "poly_ddf", "f32", nu0=0.0, sensor_A=1.5)
    assert c.stats().n_general_blocks[0] == 0
    spec = I.GridSpec(2, (256, ny), 1, [], (False, True),
                      {"x-": ("dirichlet_rho", 1.0, (0.05, 0.0, 0.0), 0.0), "x+": ("neumann",)})
    c2 = lt.Context(2, device=-1)
    c2.configure(spec, "D2Q37", "poly_ddf", "f32", nu0=0.0, sensor_A=1.5)
    assert c2.stats().n_general_blocks[0] == ny // 16
