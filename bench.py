"""Benchmark of the multi-level collide-and-stream path (one JSON line on rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--storage f32|f16dev|f64] [--no-graph]

Workload: D3Q27 recursive-regularized flow past a sphere (diameter 64 finest cells) in a
1024x512x512 finest-unit box with 4 levels (about 45 M cells, 38.9 M fine-equivalent), inflow
Mach 0.1, Re 3900, seeded 1e-3 velocity perturbation.  A step is one coarse step (8 fine
iterations, every level advanced on its schedule).  Metric: fine-equivalent MLUPS = cell updates
per second (sum over levels of cells x updates per coarse step), aggregated over ranks.

Under torchrun (N > 1) every rank runs an independent replica on its own GPU (the path has no
exchange step); the time is the max over ranks and the value the sum of their updates.

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload (the
reduced copy at 1/4 extents, sphere diameter 16, same level structure), one fine iteration per
step, on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2504_04465_b300 import inputs as I  # noqa: E402

BYTES_PER_UPDATE = {"f64": 432, "f32": 216, "f16dev": 108}   # 27 populations read + written
WORKLOAD = ("D3Q27 recursive-regularized, flow past a sphere (D = 64 finest cells), 4 levels, "
            "1024x512x512 finest-unit box, Ma 0.1, Re 3900")
CSRC = os.path.join(ROOT, "paper_2504_04465_b300", "csrc")

# Figures taken from ncu captures of the step kernels (``--counters PATH`` runs the captured
# case; the ncu command that took it is given with its summary in the repository).  Each entry records
# the kernel sources it was taken on (``source_hash``); when those files have changed since,
# the figure is reported as null instead of a stale number.
#   dram: DRAM bytes (read + write) per cell update of both step kernels over one coarse step
#         of the main workload at half extents
#   flops: executed floating-point operations per cell update (fadd + fmul + 2 ffma, packed
#          FP32 pairs 2 fadd2 + 2 fmul2 + 4 ffma2, and the same for FP64), both step kernels,
#          one coarse step of the captured case
COUNTERS = {
    ('d2q13n32:band', "flops"): {"value": 4595.7, "source_hash": '6306a43a84286b15',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2) of both step kernels over one coarse step of the 2048^2 Sod tube from t = 0.1 L / c_s, 2.07 Newton iterations per update'},
    ('d2q13n32:sqr', "flops"): {"value": 4355.5, "source_hash": '6306a43a84286b15',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2) of both step kernels over one coarse step of the 2048^2 Sod tube from t = 0.1 L / c_s, 1.92 Newton iterations per update'},
    ('d2q13n32:unif', "flops"): {"value": 3137.4, "source_hash": '6306a43a84286b15',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2) of both step kernels over one coarse step of the 2048^2 Sod tube from t = 0.1 L / c_s, 1.29 Newton iterations per update'},
    ('d2q21n32:band', "flops"): {"value": 4006.0, "source_hash": 'c6ba864d30f43d25',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2) of both step kernels over one coarse step of the 2048^2 Sod tube from t = 0.1 L / c_s, 1.15 Newton iterations per update'},
    ('d2q21n32:riemann_axes', "flops"): {"value": 2905.7, "source_hash": 'c6ba864d30f43d25',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2) of the step kernels over one coarse step of the 2D Riemann configuration 12 on the axes grid at N_c = 256 from the eighth coarse step, 0.73 Newton iterations per update'},
    ('d2q21n32:riemann_diag', "flops"): {"value": 2444.7, "source_hash": 'c6ba864d30f43d25',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2) of the step kernels over one coarse step of the 2D Riemann configuration 12 on the diag grid at N_c = 256 from the eighth coarse step, 0.54 Newton iterations per update'},
    ('d2q21n32:riemann_optim', "flops"): {"value": 2741.9, "source_hash": 'c6ba864d30f43d25',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2) of the step kernels over one coarse step of the 2D Riemann configuration 12 on the optim grid at N_c = 256 from the eighth coarse step, 0.65 Newton iterations per update'},
    ('d2q21n32:sqr', "flops"): {"value": 3778.2, "source_hash": 'c6ba864d30f43d25',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2) of both step kernels over one coarse step of the 2048^2 Sod tube from t = 0.1 L / c_s, 1.07 Newton iterations per update'},
    ('d2q21n32:unif', "flops"): {"value": 2880.1, "source_hash": 'c6ba864d30f43d25',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2) of both step kernels over one coarse step of the 2048^2 Sod tube from t = 0.1 L / c_s, 0.68 Newton iterations per update'},
    ('d2q21n64:poly', "flops"): {"value": 37858.4, "source_hash": 'e195a62c6c1fc144',
                   "capture": 'ncu, executed FP64 DADD/DMUL/DFMA thread instructions (FMA as 2) of both step kernels over one coarse step of the 5-level NACA0012 grid at chord 256, Mach 1.5, after 3 coarse steps, 11.74 Newton iterations per update'},
    ('d2q21n64:warm', "flops"): {"value": 8578.6, "source_hash": 'e195a62c6c1fc144',
                   "capture": 'ncu, executed FP64 DADD/DMUL/DFMA thread instructions (FMA as 2) of both step kernels over one coarse step of the 5-level NACA0012 grid at chord 256, Mach 1.5, after 3 coarse steps, 2.66 Newton iterations per update'},
    ('d2q21w:f32', "flops"): {"value": 546.0, "source_hash": '9de5e6796561a88c',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2) of both step kernels over one coarse step of a uniform periodic 1024^2 shear layer'},
    ('d2q37n32:band', "flops"): {"value": 6318.2, "source_hash": 'a8312b3c4a57c778',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2) of both step kernels over one coarse step of the 2048^2 Sod tube from t = 0.1 L / c_s, 1.13 Newton iterations per update'},
    ('d2q37n32:sqr', "flops"): {"value": 5964.3, "source_hash": 'a8312b3c4a57c778',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2) of both step kernels over one coarse step of the 2048^2 Sod tube from t = 0.1 L / c_s, 1.04 Newton iterations per update'},
    ('d2q37n32:unif', "flops"): {"value": 4487.5, "source_hash": 'a8312b3c4a57c778',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2) of both step kernels over one coarse step of the 2048^2 Sod tube from t = 0.1 L / c_s, 0.63 Newton iterations per update'},
    ('d2q37p:naca_f32', "flops"): {"value": 961.5, "source_hash": '93aef3942399df86',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2) of both step kernels over one coarse step of the 5-level NACA0012 grid at chord 256'},
    ('d2q37p:naca_f64', "flops"): {"value": 1361.6, "source_hash": '93aef3942399df86',
                   "capture": 'ncu, executed FP64 DADD/DMUL/DFMA thread instructions (FMA as 2) of both step kernels over one coarse step of the 5-level NACA0012 grid at chord 256'},
    ('d2q37p:sod_f32', "flops"): {"value": 1095.0, "source_hash": '93aef3942399df86',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2) of both step kernels over one coarse step of the 4096x64 Sod tube'},
    ('d2q37p:sod_f64', "flops"): {"value": 1661.2, "source_hash": '93aef3942399df86',
                   "capture": 'ncu, executed FP64 DADD/DMUL/DFMA thread instructions (FMA as 2) of both step kernels over one coarse step of the 4096x64 Sod tube'},
    ('d2q9:f32', "flops"): {"value": 243.0, "source_hash": '8883843697529bb4',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2) of both step kernels over one coarse step of a uniform periodic 2048^2 Taylor-Green grid'},
    ('d2q9:f64', "flops"): {"value": 253.0, "source_hash": '8883843697529bb4',
                   "capture": 'ncu, executed FP64 DADD/DMUL/DFMA thread instructions (FMA as 2) of both step kernels over one coarse step of a uniform periodic 2048^2 Taylor-Green grid'},
    ('d3q27:f16dev', "dram"): {"value": 113.4, "source_hash": 'b4231998c5fedfe9',
                   "capture": 'ncu, dram__bytes_read.sum + dram__bytes_write.sum of both step kernels over one coarse step of the D3Q27 sphere at half extents (512x256x256, 5.68 M cells)'},
    ('d3q27:f16dev', "flops"): {"value": 468.7, "source_hash": 'b4231998c5fedfe9',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2, packed FP32-pair FADD2/FMUL2/FFMA2 as 2/2/4) of both step kernels over one coarse step of the D3Q27 sphere at half extents (512x256x256, 5.68 M cells)'},
    ('d3q27:f32', "dram"): {"value": 225.5, "source_hash": 'b4231998c5fedfe9',
                   "capture": 'ncu, dram__bytes_read.sum + dram__bytes_write.sum of both step kernels over one coarse step of the D3Q27 sphere at half extents (512x256x256, 5.68 M cells)'},
    ('d3q27:f32', "flops"): {"value": 612.5, "source_hash": 'b4231998c5fedfe9',
                   "capture": 'ncu, executed FP32 FADD/FMUL/FFMA thread instructions (FMA as 2) of both step kernels over one coarse step of the D3Q27 sphere at half extents (512x256x256, 5.68 M cells)'},
    ('d3q27:f64', "dram"): {"value": 447.2, "source_hash": 'b4231998c5fedfe9',
                   "capture": 'ncu, dram__bytes_read.sum + dram__bytes_write.sum of both step kernels over one coarse step of the D3Q27 sphere at half extents (512x256x256, 5.68 M cells)'},
    ('d3q27:f64', "flops"): {"value": 621.8, "source_hash": 'b4231998c5fedfe9',
                   "capture": 'ncu, executed FP64 DADD/DMUL/DFMA thread instructions (FMA as 2) of both step kernels over one coarse step of the D3Q27 sphere at half extents (512x256x256, 5.68 M cells)'},
}


def source_hash(files) -> str:
    """sha256 (first 16 hex digits) of the listed kernel source files, in order."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


# the files each kernel path is compiled from (its translation unit and the headers it includes)
_COMMON = ["kernels_impl.cuh", "device_common.cuh", "device_types.h", "models.cuh", "models_comp.cuh",
           "lattice_tables.h", "kernels.h", "mlp.cuh"]
PATH_SOURCES = {
    "d3q27": ["k_d3q27.cu"] + _COMMON,
    "d2q9": ["k_d2q9.cu"] + _COMMON,
    "d2q37p": ["k_d2q37.cu", "d2q37.cuh", "weights.cpp"] + _COMMON,
    "d2q21w": ["k_d2q21w.cu"] + _COMMON,
    "d2q21n32": ["k_d2q21_n32_f32.cu", "d2q21.cuh"] + _COMMON,
    "d2q13n32": ["k_d2q13.cu", "weak_h3.cuh"] + _COMMON,
    "d2q37n32": ["k_d2q37_n32_f32.cu", "d2q37.cuh"] + _COMMON,
    "d2q21n64": ["k_d2q21.cu", "d2q21.cuh"] + _COMMON,
}


def counter(path: str, key: str):
    """(value, note) of a captured figure, value None when missing or taken on other sources."""
    e = COUNTERS.get((path, key))
    if e is None:
        return None, "not captured"
    if e["source_hash"] != source_hash(PATH_SOURCES[path.split(":")[0]]):
        return None, "kernel sources changed since the capture"
    return e["value"], e["capture"]


def peaks():
    """Measured HBM copy bandwidth of the B300s (GB/s) and where it comes from."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


_PIPE = {}


def pipe_peaks(device: int) -> dict:
    """Measured FP32, packed-FP32 and FP64 FMA throughput of this GPU (TFLOP/s), once per run."""
    if not _PIPE:
        from paper_2504_04465_b300 import lbmtree as lt
        for k in ("fp32", "fp32x2", "fp64"):
            _PIPE[k] = lt.pipe_peak(k, device, 8192)[0] / 1e12
        _PIPE["how"] = ("lbm_pipe_peak: one wave of 256-thread blocks, 8 independent FMA chains per thread, "
                        "best of 5 launches; fp32x2 = packed fma.rn.f32x2, the FP32 lanes' limit")
    return _PIPE


def roofline(updates: float, ms: float, bytes_per_update: float, pipe: str | None, flops_path: str | None,
             device: int) -> dict:
    """HBM and pipe fractions of a timed path: achieved bytes (algorithmic, per update) and
    executed flops (captured, per update) over the event-timed duration, against the measured
    HBM copy bandwidth and the measured pipe peak; frac is the larger of the two (the roofline
    is the slower of the two limits)."""
    hbm, kind = peaks()
    gbs = bytes_per_update * updates / (ms * 1e-3) / 1e9
    out = {"bytes_per_update": bytes_per_update, "achieved_gbs": gbs, "hbm_peak_gbs": hbm, "hbm_peak_kind": kind,
           "hbm_frac": gbs / hbm}
    frac, bound = gbs / hbm, "hbm"
    if pipe:
        fpu, note = counter(flops_path, "flops") if flops_path else (None, "not captured")
        pk = pipe_peaks(device)["fp32x2" if pipe == "fp32" else "fp64"]
        out.update({"pipe": pipe, "flops_per_update": fpu, "flops_source": note, "pipe_peak_tflops": pk})
        if fpu is not None:
            tf = fpu * updates / (ms * 1e-3) / 1e12
            out.update({"achieved_tflops": tf, "pipe_frac": tf / pk})
            if tf / pk > frac:
                frac, bound = tf / pk, pipe
    out.update({"frac": frac, "bound": bound})
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def replica_totals(ms: float, updates: int, dist=None, device: str = "cpu"):
    """Whole-job figures of independent replicas: the slowest rank's time and the sum of the
    ranks' cell updates (value = updates / time)."""
    if dist is None:
        return ms, updates
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    n = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(float(n.item())))


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# block shape and step-kernel variant picked by paper_2504_04465_b300.autotune on a B300 for this
# workload (overridable with --block / --variant, or re-tuned with --autotune)
DEFAULT_BLOCK = {"f32": (8, 4, 4), "f16dev": (8, 4, 4), "f64": (8, 4, 4)}
DEFAULT_VARIANT = {"f32": 1, "f16dev": 1, "f64": 0}


def make_context(spec, storage, device, stream, graph, scale=1, block=None, variant=0):
    from paper_2504_04465_b300 import lbmtree as lt
    ctx = lt.Context(3, device=device, stream=stream)
    ctx.configure(spec, "D3Q27", "rr", storage, block=block, nu0=I.sphere_nu0(scale))
    if variant:
        ctx.set_variant(variant)
    if graph:
        ctx.use_graph(True)
    return ctx


def host_fields(ctx):
    lv, xyz, _ = ctx.cells()
    n = lv.size
    rho = np.ones(n)
    u = np.zeros((3, n))
    for level in np.unique(lv):
        m = lv == level
        r, uu = I.sphere_fields(int(level), xyz[m])
        rho[m] = r
        u[:, m] = uu
    return rho, u


def cpu_sample(n_fine: int):
    """Oracle on the reduced sphere workload: (MLUPS, seconds, cell updates)."""
    from oracle import grid as G
    from oracle import lattices as L
    from oracle import solver as S
    g = G.build(I.sphere_spec(4), L.D3Q27)
    s = S.Solver(g, "rr", nu0=I.sphere_nu0(4))
    s.init_fields([(*I.sphere_fields(lv.level, lv.coords), None) for lv in g.levels])
    counts = [int((lv.ctype != G.SOLID).sum()) for lv in g.levels]
    return s, counts


def oracle_updates(counts, t0, n):
    """Cell updates of fine iterations t0 .. t0+n-1 (level i updates when t % 2^i == 0)."""
    return sum(c for t in range(t0, t0 + n) for i, c in enumerate(counts) if t % (1 << i) == 0)


def _cpu_worker(seconds: float):
    """One oracle replica on the reduced sphere for about ``seconds``: (cell updates, seconds)."""
    s, counts = cpu_sample(0)
    t0 = time.perf_counter()
    nf = 0
    while time.perf_counter() - t0 < seconds:
        s.fine_iteration()
        nf += 1
    return oracle_updates(counts, 0, nf), time.perf_counter() - t0, nf


def cpu_baseline(seconds: float, max_workers: int = 32) -> dict:
    """The oracle on the host cores: one process, then independent replicas in a process pool
    (spawned, one single-threaded worker per core up to max_workers), whole-pool updates over
    the pool's wall time."""
    import multiprocessing as mp
    upd, dt, nf = _cpu_worker(seconds)
    one = {"value": upd / dt / 1e6, "unit": "MLUPS", "cores": 1,
           "sample": f"{nf} fine iterations in {dt:.1f} s"}
    n = max(1, min(os.cpu_count() or 1, max_workers))
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(n) as pool:
            res = pool.map(_cpu_worker, [seconds] * n)
        wall = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    tot = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    return {"value": tot / busy / 1e6, "unit": "MLUPS", "cores": n, "kind": "oracle",
            "sample": (f"FP64 numpy oracle, reduced sphere workload (256x128x128, D=16, 4 levels): {n} independent "
                       f"single-threaded replicas in a spawned process pool ({os.cpu_count()} host cores, at most "
                       f"{max_workers} workers), {sum(r[2] for r in res)} fine iterations in all, updates over the "
                       f"slowest replica's {busy:.1f} s (pool wall time with start-up {wall:.1f} s)"),
            "one_core": one}


def run_reference(args, world, rank):
    if rank != 0:
        return
    s, counts = cpu_sample(0)
    for _ in range(args.warmup):
        s.fine_iteration()
    t0 = s.t
    start = time.perf_counter()
    for _ in range(args.steps):
        s.fine_iteration()
    dt = time.perf_counter() - start
    upd = oracle_updates(counts, t0, args.steps)
    v = upd / dt / 1e6
    sample = (f"FP64 numpy oracle, reduced sphere workload (256x128x128, sphere D=16, 4 levels, "
              f"{sum(counts)} cells), {args.steps} fine iterations after {args.warmup} warm-up")
    line = {"impl": "reference", "metric": "fine-equivalent MLUPS", "value": v, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "reduced copy at 1/4 extents", "step": "one fine iteration"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ cases of the kernel paths
def _init_ctx(ctx, fields):
    """Initial fields from fields(level, coords) -> (rho, u[, T]) at every listed cell."""
    lv, xyz, _ = ctx.cells()
    n, D = lv.size, ctx.dim
    rho, u, T = np.ones(n), np.zeros((D, n)), np.zeros(n)
    comp = False
    for L in np.unique(lv):
        m = lv == L
        r = fields(int(L), xyz[m, :D])
        rho[m], u[:, m] = r[0], r[1]
        if len(r) > 2:
            T[m], comp = r[2], True
    ctx.init_fields(rho, u, T if comp else None)


def sod_numerical_case(lat, grid, L, stream, local):
    """The Sec. 7.6 Sod benchmark case (numerical equilibrium, FP32 populations and FP32 Newton)."""
    from paper_2504_04465_b300 import lbmtree as lt
    grids = {"unif": I.sod_spec(L, L), "band": I.sod_spec(L, L, 2, (L // 4, 3 * L // 4)),
             "sqr": I.GridSpec(2, (L, L), 2, [(0, (L // 4, L // 4), (3 * L // 4, 3 * L // 4))], (False, True),
                               {"x-": ("neumann",), "x+": ("neumann",)})}
    T0 = {"D2Q13": 0.35, "D2Q21": 0.9, "D2Q37": 1.0}[lat]   # inviscid reference temperatures of Sec. 6
    ctx = lt.Context(2, device=local, stream=stream)
    ctx.configure(grids[grid], lat, "num_ddf", "f32", nu0=0.0, T0=T0, sensor_A=1.5, newton_fp32=True)
    _init_ctx(ctx, lambda lev, c: I.sod_fields(I.cell_centres(c, lev), L, T0))
    # the timed window starts once the three waves have formed: t = 0.1 L / c_s (finest units)
    fine = int(0.1 * L / np.sqrt(1.4 * T0))
    return ctx, T0, fine


def riemann12_case(grid, nc, stream, local):
    """Sec. 6.2's 2D Riemann problem, configuration 12: D2Q21 DDF with the numerical equilibrium,
    FP32 populations and FP32 Newton, inviscid with the kinetic sensor (A = 1.5), periodic, on the
    diag, axes or optim grid with nc coarse cells per half side L."""
    from paper_2504_04465_b300 import lbmtree as lt
    T0 = 0.9
    ctx = lt.Context(2, device=local, stream=stream)
    ctx.configure(I.riemann12_spec(nc, grid), "D2Q21", "num_ddf", "f32", nu0=0.0, T0=T0, sensor_A=1.5,
                  newton_fp32=True)
    _init_ctx(ctx, lambda lev, c: I.riemann12_fields(I.cell_centres(c, lev), nc, T0))
    return ctx


def naca37_case(chord, storage, stream, local, n_levels=5):
    """BASELINE configuration 3b: D2Q37 polynomial DDF around a NACA0012 at zero incidence,
    Mach 0.8 subsonic inlet (density extrapolated), Re 1e4 on the chord, sensor A = 1.35."""
    from paper_2504_04465_b300 import lbmtree as lt
    mach, T0, gamma = 0.8, lt.lattice_cs2("D2Q37"), 1.4
    spec = I.naca_spec(chord, mach, T0, gamma, n_levels=n_levels, supersonic=False)
    ctx = lt.Context(2, device=local, stream=stream)
    ctx.configure(spec, "D2Q37", "poly_ddf", storage, nu0=mach * np.sqrt(gamma * T0) * chord / 1e4, gamma=gamma,
                  sensor_A=1.35)
    _init_ctx(ctx, lambda lev, c: I.naca_fields(lev, c, mach, T0, gamma))
    return ctx


def counters_case(path, stream, local):
    """(context, coarse steps before the counted step) of a captured kernel path."""
    from paper_2504_04465_b300 import lbmtree as lt
    fam, case = path.split(":")
    if fam == "d3q27":
        ctx = make_context(I.sphere_spec(2), case, local, stream, False, 2, DEFAULT_BLOCK[case], DEFAULT_VARIANT[case])
        ctx.init_fields(*host_fields(ctx))
        return ctx, 3
    if fam == "d2q9":
        ctx = lt.Context(2, device=local, stream=stream)
        ctx.configure(I.taylor_green_spec(2048, 0, 0, 1), "D2Q9", "rr", case, nu0=0.01)
        _init_ctx(ctx, lambda lev, c: I.taylor_green_fields(I.cell_centres(c, lev), 2048, 1, 0.05, 1.0 / 3.0))
        return ctx, 3
    if fam == "d2q37p":
        geom, st = case.split("_")
        if geom == "sod":
            ctx = lt.Context(2, device=local, stream=stream)
            ctx.configure(I.sod_spec(4096, 64), "D2Q37", "poly_ddf", st, nu0=0.0, sensor_A=1.5)
            T0 = lt.lattice_cs2("D2Q37")
            _init_ctx(ctx, lambda lev, c: I.sod_fields(I.cell_centres(c, lev), 4096, T0))
            return ctx, 3
        return naca37_case(256, st, stream, local), 3
    if fam == "d2q21w":
        n = 1024
        ctx = lt.Context(2, device=local, stream=stream)
        ctx.configure(I.GridSpec(2, (n, n), 1, [], (True, True)), "D2Q21", "rr", case, nu0=0.01)
        _init_ctx(ctx, lambda lev, c: (np.ones(c.shape[0]), np.stack(
            [0.05 * np.sin(2 * np.pi * I.cell_centres(c, lev)[:, 1] / n), np.zeros(c.shape[0])])))
        return ctx, 3
    if fam == "d2q21n32" and case.startswith("riemann_"):
        return riemann12_case(case[len("riemann_"):], 256, stream, local), 8
    if fam in ("d2q13n32", "d2q21n32", "d2q37n32"):
        lat = {"d2q13n32": "D2Q13", "d2q21n32": "D2Q21", "d2q37n32": "D2Q37"}[fam]
        ctx, _, fine = sod_numerical_case(lat, case, 2048, stream, local)
        return ctx, max(3, fine // (2 ** (ctx.stats().n_levels - 1)))
    if fam == "d2q21n64":
        P = dict(LEARNED, chord=256)
        spec = I.naca_spec(P["chord"], P["mach"], P["T0"], P["gamma"])
        u_in = P["mach"] * np.sqrt(P["gamma"] * P["T0"])
        ctx = lt.Context(2, device=local, stream=stream)
        ctx.configure(spec, "D2Q21", "num_ddf", "f32", nu0=u_in * P["chord"] / P["Re"], T0=P["T0"], gamma=P["gamma"],
                      sensor_A=P["sensor_A"], guess=case)
        _init_ctx(ctx, lambda lev, c: I.naca_fields(lev, c, P["mach"], P["T0"], P["gamma"]))
        return ctx, 3
    raise ValueError(path)


def run_counters(args, local):
    """Run one captured kernel path: warm-up coarse steps, then one coarse step inside the NVTX
    range "timed" (no graph, so an ncu capture filtered on that range sees each launch)."""
    import torch
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    ctx, pre = counters_case(args.counters, stream.cuda_stream, local)
    ctx.step(pre)
    torch.cuda.synchronize()
    s0 = ctx.stats()
    from paper_2504_04465_b300 import lbmtree as lt
    torch.cuda.nvtx.range_push("timed")
    ctx.step(1)
    try:
        ctx.sync()
    except lt.LbmError as e:                 # solves stopped unconverged: the step completed
        if lt.ERR.get(e.code) != "NEWTON":
            raise
    torch.cuda.nvtx.range_pop()
    s1 = ctx.stats()
    it = (s1.newton_iter_sum - s0.newton_iter_sum) / max(1, s1.newton_updates - s0.newton_updates)
    print(json.dumps({"counters": args.counters, "cell_updates": int(s1.cell_updates),
                      "launches": int(s1.kernel_launches - s0.kernel_launches), "newton_iterations": it,
                      "source_hash": source_hash(PATH_SOURCES[args.counters.split(":")[0]])}), flush=True)
    ctx.close()


# ------------------------------------------------------------------ forms beside the plain FP32 method
def _event_ms(stream, fn, reps=1):
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(reps):
            fn()
        ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / reps


def _moment_err(a, b, types):
    """Relative L2 of rho and u of context a against context b over the listed cell types."""
    ra, ua, _ = a.moments()
    rb, ub, _ = b.moments()
    m = np.isin(types, (1, 4))
    return {"rho": float(np.linalg.norm(ra[m] - rb[m]) / np.linalg.norm(rb[m])),
            "u": float(np.linalg.norm(ua[:, m] - ub[:, m]) / np.linalg.norm(ub[:, m]))}


def form_fp16(args, stream, local, f32_ms):
    """FP16-deviation storage on the same workload, and its error after 20 coarse steps on the
    reduced sphere against the FP64 GPU path (itself equal to the oracle within 1e-12)."""
    ctx = make_context(I.sphere_spec(args.scale), "f16dev", local, stream.cuda_stream, True, args.scale,
                       DEFAULT_BLOCK["f16dev"], DEFAULT_VARIANT["f16dev"])
    ctx.init_fields(*host_fields(ctx))
    ctx.step(args.warmup)
    upd = ctx.stats().cell_updates
    ms = _event_ms(stream, lambda: ctx.step(args.steps)) / args.steps
    ctx.sync()
    ctx.close()
    errs = {}
    ref = make_context(I.sphere_spec(4), "f64", local, stream.cuda_stream, True, 4, (8, 4, 4), 0)
    ref.init_fields(*host_fields(ref))
    ref.step(20)
    types = ref.cells()[2]
    for st in ("f32", "f16dev"):
        c = make_context(I.sphere_spec(4), st, local, stream.cuda_stream, True, 4, (8, 4, 4), 0)
        c.init_fields(*host_fields(c))
        c.step(20)
        errs[st] = _moment_err(c, ref, types)
        c.close()
    ref.close()
    return {"workload": "same as the main line, populations stored as binary16 deviations from w rho_ref",
            "ms_per_step": ms, "value": upd / ms / 1e3, "unit": "MLUPS", "speedup_vs_f32": f32_ms / ms,
            "roofline": roofline(upd, ms, BYTES_PER_UPDATE["f16dev"], "fp32", "d3q27:f16dev", local),
            "err_vs_f64": errs,
            "err_case": "reduced sphere (256x128x128, D=16, 4 levels), 20 coarse steps, relative L2 over bulk and "
                        "boundary cells against the FP64 path"}


LEARNED = {"chord": 2304, "mach": 1.5, "T0": 0.65, "Re": 1e4, "gamma": 1.4, "sensor_A": 1.35}


def form_learned(args, stream, local):
    """Numerical-equilibrium D2Q21 flow past a NACA0012 at Mach 1.5 (5 levels, N_eq 7.9 M):
    Newton from the polynomial guess (the plain method), from the network trained here on the
    solver's own equilibria, and from the previous multipliers (warm start)."""
    import torch
    from paper_2504_04465_b300 import lbmtree as lt
    P = dict(LEARNED)
    if args.scale > 1:
        P["chord"] = 256
    spec = I.naca_spec(P["chord"], P["mach"], P["T0"], P["gamma"])
    u_in = P["mach"] * np.sqrt(P["gamma"] * P["T0"])
    ctx = lt.Context(2, device=local, stream=stream.cuda_stream)
    ctx.configure(spec, "D2Q21", "num_ddf", "f32", nu0=u_in * P["chord"] / P["Re"], T0=P["T0"], gamma=P["gamma"],
                  sensor_A=P["sensor_A"], guess="warm")
    lv, xyz, ty = ctx.cells()
    n = lv.size
    rho, u, T = np.ones(n), np.zeros((2, n)), np.full(n, P["T0"])
    for L in np.unique(lv):
        m = lv == L
        r, uu, tt = I.naca_fields(int(L), xyz[m, :2], P["mach"], P["T0"], P["gamma"])
        rho[m], u[:, m], T[m] = r, uu, tt
    ctx.init_fields(rho, u, T)
    ctx.step(3)                                        # leave the impulsive start (warm start)
    # training samples: (u, T) of the solver's fluid cells, filtered, split 90/10; targets are
    # the converged multipliers at exactly those states (batched Newton from lambda = 0)
    rho, u, T = ctx.moments()
    cs = np.sqrt(P["gamma"] * P["T0"])
    keep = (ty == 1) & (T > 0.5 * P["T0"]) & (T < 2 * P["T0"]) & (np.sqrt((u ** 2).sum(0)) < 2 * cs)
    idx = np.random.default_rng(1504).permutation(np.nonzero(keep)[0])[:1_000_000]
    ntr = int(0.9 * idx.size)
    d_uT = torch.tensor(np.stack([u[0, idx], u[1, idx], T[idx]], axis=1), device="cuda")
    d_lam = torch.empty((idx.size, 8), dtype=torch.float64, device="cuda")
    d_it = torch.empty(idx.size, dtype=torch.int32, device="cuda")
    ctx.newton_batch(d_uT.data_ptr(), idx.size, "zero", d_lam.data_ptr(), d_it.data_ptr())
    ctx.sync()
    lam_ref = d_lam.cpu().numpy()
    train = {}
    for tc in (False, True):          # FP32 cores, then BF16 tensor cores (the network kept)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss = ctx.mlp_train(d_uT.data_ptr(), d_lam.data_ptr(), ntr, steps=3000, batch=4096, lr=3e-3, lr_final=3e-4,
                             seed=1504, tensor_cores=tc)
        torch.cuda.synchronize()
        train["tensor_cores" if tc else "fp32_cores"] = {"seconds": time.perf_counter() - t0, "final_loss": loss}
    train_s = train["tensor_cores"]["seconds"]
    held = {}
    nte = idx.size - ntr
    d_te = d_uT[ntr:].contiguous()
    for g in ("zero", "poly", "mlp"):
        d_l = torch.empty((nte, 8), dtype=torch.float64, device="cuda")
        d_i = torch.empty(nte, dtype=torch.int32, device="cuda")
        ctx.newton_batch(d_te.data_ptr(), nte, g, d_l.data_ptr(), d_i.data_ptr())
        ctx.sync()
        it = d_i.cpu().numpy()
        held[g] = {"mean_iters": float(it[it >= 0].mean()) if (it >= 0).any() else None,
                   "nonconverged": int((it < 0).sum()),
                   "max_abs_dlambda_vs_zero_guess": float(np.abs(d_l.cpu().numpy() - lam_ref[ntr:]).max())}
    def timed_runs(K, tune, fp64):
        out = {}
        for g in ("poly", "mlp", "warm"):
            ctx.set_guess(g)
            ctx.step(1)
            v = ctx.autotune(1)[0] if tune else 0     # occupancy variant for this guess
            s0 = ctx.stats()
            ms = _event_ms(stream, lambda: ctx.step(K)) / K
            ctx.sync()
            s1 = ctx.stats()
            out[g] = {"ms_per_step": ms, "value": s1.cell_updates / ms / 1e3, "unit": "MLUPS",
                      "mean_newton_iters": (s1.newton_iter_sum - s0.newton_iter_sum) /
                      max(1, s1.newton_updates - s0.newton_updates),
                      "nonconverged": s1.newton_nonconverged - s0.newton_nonconverged,
                      "variant_min_blocks": ctx.variants()[v],
                      "roofline": roofline(s1.cell_updates, ms, 464, "fp64" if fp64 else "fp32",
                                           f"d2q21n64:{g}" if fp64 else None, local)}
        return out

    runs = timed_runs(1, False, True)
    # the same comparison with the solve on the FP32 pipe (tolerance 1e-5)
    ctx.set_newton_precision(True, 1e-5)
    try:
        runs32 = timed_runs(3, True, False)
        fp32 = {"tol": 1e-5, "by_guess": runs32,
                "speedup_mlp_vs_poly": runs32["poly"]["ms_per_step"] / runs32["mlp"]["ms_per_step"],
                "speedup_vs_fp64_warm": runs["warm"]["ms_per_step"] / runs32["warm"]["ms_per_step"]}
    except Exception as e:                      # a solve that did not converge sets the status
        fp32 = {"error": f"{type(e).__name__}: {e}"}
    st = ctx.stats()
    ctx.close()
    return {"workload": f"D2Q21 numerical equilibrium, NACA0012 chord {P['chord']}, Mach {P['mach']}, T0 {P['T0']}, "
                        f"Re {P['Re']:.0f}, 5 levels, N_eq {st.n_eq:.0f}, FP32 populations, FP64 Newton (tol 1e-12)",
            "step": "one coarse step = 16 fine iterations", "by_guess": runs,
            "speedup_mlp_vs_poly": runs["poly"]["ms_per_step"] / runs["mlp"]["ms_per_step"],
            "iterations_saved_vs_poly": runs["poly"]["mean_newton_iters"] - runs["mlp"]["mean_newton_iters"],
            "fp32_newton": fp32,
            "heldout_newton": held,
            "training": {"samples": int(ntr), "heldout": int(nte), "steps": 3000, "batch": 4096, "final_loss": loss,
                         "seconds": train_s, "by_path": train,
                         "speedup_tensor_cores": train["fp32_cores"]["seconds"] / train["tensor_cores"]["seconds"],
                         "network_used": "the tensor-core trained one",
                         "filter": "T in [0.5, 2] T0, |u| < 2 sqrt(gamma T0), fluid cells"},
            "err": "Newton runs to the same tolerance from every guess: results agree within it"}


def form_d2q37(args, stream, local):
    """D2Q37 polynomial-equilibrium DDF with the shock sensor on Sod tubes (inviscid, A = 1.5):
    the 4096x64 tube uniform and with its middle half refined (2 levels), and a 16384x512 tube
    for a bandwidth-sized case; FP32 and FP64 populations."""
    from paper_2504_04465_b300 import lbmtree as lt
    out = {"workload": "Sod shock tube (rho, p) = (1, 1) | (0.125, 0.1), T = T0 p / rho, T0 = c_s^2 of D2Q37, "
                       "Neumann ends, periodic across, inviscid with the kinetic sensor (A = 1.5)",
           "bytes_per_update": {"f32": 592, "f64": 1184},
           "flops_note": "flops per update captured on the 4096x64 tube"}
    cases = {"4096x64": I.sod_spec(4096, 64), "4096x64_band": I.sod_spec(4096, 64, 2, (1024, 3072)),
             "16384x512": I.sod_spec(16384, 512)}
    for name, spec in cases.items():
        for st in ("f32", "f64"):
            ctx = lt.Context(2, device=local, stream=stream.cuda_stream)
            ctx.configure(spec, "D2Q37", "poly_ddf", st, nu0=0.0, sensor_A=1.5)
            ctx.use_graph(True)
            lv, xyz, _ = ctx.cells()
            from paper_2504_04465_b300.lbmtree import lattice_cs2
            T0 = lattice_cs2("D2Q37")
            rho, u, T = I.sod_fields(I.cell_centres(xyz[:, :2], lv), spec.extent[0], T0)
            ctx.init_fields(rho, u, T)
            ctx.step(2)
            upd = ctx.stats().cell_updates
            K = 20
            ms = _event_ms(stream, lambda: ctx.step(K)) / K
            ctx.sync()
            bpu = 592 if st == "f32" else 1184
            out[f"{name}_{st}"] = {"ms_per_step": ms, "value": upd / ms / 1e3, "unit": "MLUPS",
                                   "roofline": roofline(upd, ms, bpu, "fp32" if st == "f32" else "fp64",
                                                        f"d2q37p:sod_{st}", local)}
            ctx.close()
    return out


def form_d2q21_weak(args, stream, local):
    """Weakly compressible D2Q21 (Hermite basis to order 3) on a periodic shear layer, uniform
    4096^2 (--scale divides the side): RR and BGK, FP32 deviations."""
    from paper_2504_04465_b300 import lbmtree as lt
    n = 4096 // args.scale
    spec = I.GridSpec(2, (n, n), 1, [], (True, True))
    out = {"workload": f"D2Q21 weakly compressible, periodic {n}x{n}, u_x = 0.05 sin(2 pi y / L), rho = 1, "
                       "nu0 = 0.01", "bytes_per_update": 168, "unit": "MLUPS",
           "flops_note": "flops per update captured on the RR model at 1024^2"}
    for model in ("rr", "bgk"):
        ctx = lt.Context(2, device=local, stream=stream.cuda_stream)
        ctx.configure(spec, "D2Q21", model, "f32", nu0=0.01)
        ctx.use_graph(True)
        lv, xyz, _ = ctx.cells()
        y = I.cell_centres(xyz[:, :2], lv)[:, 1]
        u = np.stack([0.05 * np.sin(2 * np.pi * y / n), np.zeros_like(y)])
        ctx.init_fields(np.ones(y.size), u)
        ctx.step(3)
        K = 20
        ms = _event_ms(stream, lambda: ctx.step(K)) / K
        ctx.sync()
        upd = ctx.stats().cell_updates
        out[model] = {"ms_per_step": ms, "value": upd / ms / 1e3,
                      "roofline": roofline(upd, ms, 168, "fp32", "d2q21w:f32" if model == "rr" else None, local)}
        ctx.close()
    return out


def form_sod_numerical(args, stream, local):
    """The paper's compressible performance benchmark (Sec. 7.6, Sod tube, L = 2^13, single
    precision): D2Q21 and D2Q37 DDF with the numerical equilibrium (8 constraints), FP32
    populations and FP32 Newton (tolerance 1e-5, warm start), inviscid with the kinetic sensor
    (A = 1.5), on the L x L domain uniform and with the refinement patches of Sec. 6.1 (band:
    x/L in [1/4, 3/4); sqr: a centred square of side L/2; hori: the half y/L < 1/2, whose
    interface meets the Neumann faces, which the grid builder refuses); L counts finest cells.
    The timed window starts after t = 0.1 L / c_s, once the rarefaction, contact and shock have
    formed (the paper times whole runs; the first steps of the tube, nearly at rest, need almost
    no Newton iterations and would flatter the solver)."""
    L = 8192 // args.scale                        # --scale 4: the 2048^2 profiling case
    out = {"workload": f"Sod shock tube on {L}x{L} (finest cells), (rho, p) = (1, 1) | (0.125, 0.1), "
                       "T = T0 p / rho, Neumann ends, periodic across, inviscid, kinetic sensor A = 1.5",
           "storage": "f32", "newton": "fp32, tol 1e-5, warm start", "unit": "MLUPS (cell updates per second)",
           "bytes_per_update": {"D2Q13": 336, "D2Q21": 464, "D2Q37": 720},
           "bytes_note": "f and g FP32 read and written, the eight FP64 multipliers read and written",
           "flops_note": "flops per update captured on the 2048^2 tube in the same window"}
    from paper_2504_04465_b300 import lbmtree as lt
    for lat in (("D2Q13", "D2Q21", "D2Q37") if args.sod_lattices == "all" else args.sod_lattices.split(",")):
        for gname in (args.sod_grids.split(",")):
            ctx, T0, fine = sod_numerical_case(lat, gname, L, stream.cuda_stream, local)
            ctx.use_graph(True)
            nl = ctx.stats().n_levels
            ctx.step(max(1, fine // 2 ** (nl - 1)))     # to t = 0.1 L / c_s
            v, tune_ms = ctx.autotune(2)                # occupancy variant of the step kernels
            st0 = ctx.stats()
            K = 4
            ms = _event_ms(stream, lambda: ctx.step(K)) / K
            status = "converged"
            try:
                ctx.sync()
            except lt.LbmError as e:
                if lt.ERR.get(e.code) != "NEWTON":
                    raise
                # solves stopped at their last finite iterate (states outside the lattice's
                # realisable domain: the D2Q13 rarefaction); the step itself completed
                status = "some solves stopped unconverged"
            st1 = ctx.stats()
            upd = st1.cell_updates
            it = (st1.newton_iter_sum - st0.newton_iter_sum) / max(1, st1.newton_updates - st0.newton_updates)
            fam = {"D2Q13": "d2q13n32", "D2Q21": "d2q21n32", "D2Q37": "d2q37n32"}[lat]
            out[f"{lat}_{gname}"] = {"cells": int(sum(st1.n_cells[:nl])), "ms_per_step": ms, "value": upd / ms / 1e3,
                                     "window_start_fine_iteration": int(st0.fine_iterations),
                                     "newton_iterations": it, "nonconverged": int(st1.newton_nonconverged),
                                     "newton_status": status,
                                     "variant_min_blocks": ctx.variants()[v],
                                     "autotune_ms": dict(zip(map(str, ctx.variants()), tune_ms)),
                                     "roofline": roofline(upd, ms, {"D2Q13": 336, "D2Q21": 464, "D2Q37": 720}[lat],
                                                          "fp32", f"{fam}:{gname}", local)}
            ctx.close()
    out["paper_a100"] = {"note": "Sec. 7.6 table, A100-SXM4, other machine: context only",
                         "D2Q13": {"unif": 1259.1, "hori": 1088.4, "band": 1244.8, "sqr": 1072.7},
                         "D2Q21": {"unif": 618.5, "hori": 555.9, "band": 588.2, "sqr": 544.4},
                         "D2Q37": {"unif (L = 2^12)": 286.9, "hori": 263.0, "band": 307.4, "sqr": 266.1}}
    return out


def form_riemann12(args, stream, local):
    """Sec. 6.2's 2D Riemann problem (configuration 12) at the paper's finest resolution, N_c = 512
    coarse cells per L on [-L, L]^2 (2048^2 finest cells), D2Q21 numerical DDF in FP32 with the
    FP32 Newton, on the three grids; the timed window starts at t = 0.05 t_c (t_c = L / u_0),
    once the four shocks and contacts have left the quadrant edges."""
    nc = 512 // args.scale
    T0 = 0.9
    out = {"workload": f"2D Riemann configuration 12 on [-L, L]^2, N_c = {nc} (finest {4 * nc}^2), periodic, "
                       "inviscid, kinetic sensor A = 1.5",
           "storage": "f32", "newton": "fp32, tol 1e-5, warm start", "unit": "MLUPS (cell updates per second)",
           "bytes_per_update": 464, "step": "one coarse step = 2 fine iterations"}
    from paper_2504_04465_b300 import lbmtree as lt
    for gname in ("diag", "axes", "optim"):
        ctx = riemann12_case(gname, nc, stream.cuda_stream, local)
        ctx.use_graph(True)
        ctx.step(max(1, int(0.05 * nc / np.sqrt(1.4 * T0))))     # coarse steps to t = 0.05 t_c
        v, tune_ms = ctx.autotune(2)
        st0 = ctx.stats()
        K = 4
        ms = _event_ms(stream, lambda: ctx.step(K)) / K
        ctx.sync()
        st1 = ctx.stats()
        upd = st1.cell_updates
        it = (st1.newton_iter_sum - st0.newton_iter_sum) / max(1, st1.newton_updates - st0.newton_updates)
        out[gname] = {"cells": [int(n) for n in st1.n_cells[:st1.n_levels]], "ms_per_step": ms,
                      "value": upd / ms / 1e3, "window_start_fine_iteration": int(st0.fine_iterations),
                      "newton_iterations": it, "nonconverged": int(st1.newton_nonconverged),
                      "variant_min_blocks": ctx.variants()[v],
                      "roofline": roofline(upd, ms, 464, "fp32", f"d2q21n32:riemann_{gname}", local)}
        ctx.close()
    return out


def form_naca37(args, stream, local):
    """BASELINE configuration 3b: D2Q37 polynomial DDF with the sensor around a NACA0012 at
    Mach 0.8 and Re 1e4 on 5 levels (chord 2048 finest cells, Sec. 6.3's transonic airfoil),
    FP32 against FP64 populations."""
    chord = 2048 // args.scale
    out = {"workload": f"D2Q37 polynomial DDF, NACA0012 chord {chord} finest cells, zero incidence, Mach 0.8 "
                       "(density extrapolated at the inlet), Re 1e4, sensor A = 1.35, 5 levels in [-15C, 15C]^2",
           "step": "one coarse step = 16 fine iterations", "bytes_per_update": {"f32": 592, "f64": 1184},
           "flops_note": "flops per update captured on the same grid at chord 256"}
    for st in ("f32", "f64"):
        ctx = naca37_case(chord, st, stream.cuda_stream, local)
        ctx.use_graph(True)
        ctx.step(2)
        st0 = ctx.stats()
        K = 4 if st == "f32" else 2
        ms = _event_ms(stream, lambda: ctx.step(K)) / K
        ctx.sync()
        upd = st0.cell_updates
        out[st] = {"cells": int(sum(st0.n_cells[:st0.n_levels])), "n_eq": st0.n_eq, "ms_per_step": ms,
                   "value": upd / ms / 1e3, "unit": "MLUPS",
                   "roofline": roofline(upd, ms, 592 if st == "f32" else 1184, "fp32" if st == "f32" else "fp64",
                                        f"d2q37p:naca_{st}", local)}
        ctx.close()
    out["speedup_f32_vs_f64"] = out["f64"]["ms_per_step"] / out["f32"]["ms_per_step"]
    return out


def form_d2q9(args, stream, local):
    """D2Q9 recursive regularization on large periodic Taylor-Green domains (the paper's tree
    benchmarks are D2Q9 at 2^13 x 2^13): a uniform 8192^2 grid and a 4096^2 coarse grid with its
    central half refined once; FP32 and FP64 populations."""
    from paper_2504_04465_b300 import lbmtree as lt
    out = {"bytes_per_update": {"f32": 72, "f64": 144}, "flops_note": "flops per update captured on a uniform 2048^2 grid"}
    s = 1 if args.scale == 1 else 4
    cases = {f"uniform_{8192 // s}": (I.taylor_green_spec(8192 // s, 0, 0, 1), 8192 // s, 1),
             f"two_level_{4096 // s}": (I.taylor_green_spec(4096 // s, 1024 // s, 3072 // s, 2), 4096 // s, 2)}
    for name, (spec, nc, levels) in cases.items():
        for st in ("f32", "f64"):
            ctx = lt.Context(2, device=local, stream=stream.cuda_stream)
            ctx.configure(spec, "D2Q9", "rr", st, nu0=0.01 * 2 ** (levels - 1))
            ctx.use_graph(True)
            lv, xyz, _ = ctx.cells()
            rho, u = I.taylor_green_fields(I.cell_centres(xyz[:, :2], lv), nc, levels, 0.05, 1.0 / 3.0)
            ctx.init_fields(rho, u)
            ctx.step(4)
            upd = ctx.stats().cell_updates
            K = 20
            ms = _event_ms(stream, lambda: ctx.step(K)) / K
            ctx.sync()
            bpu = 72 if st == "f32" else 144
            out[f"{name}_{st}"] = {"cells": int(lv.size), "ms_per_step": ms, "value": upd / ms / 1e3, "unit": "MLUPS",
                                   "roofline": roofline(upd, ms, bpu, "fp32" if st == "f32" else "fp64", f"d2q9:{st}",
                                                        local)}
            ctx.close()
    return out


def form_aa(args, stream, local):
    """AA-pattern in-place streaming against the two-buffer path on the same single-level
    workloads: a periodic D3Q27 RR box (512 x 256 x 256 at scale 1, perturbed uniform flow) and a
    D2Q9 RR Taylor-Green square (8192^2), FP32; updates per second, HBM fraction and device
    memory of each, and the largest D3Q27 FP32 box that fits the GPU's free memory with each."""
    import torch
    from paper_2504_04465_b300 import lbmtree as lt
    s = 1 if args.scale == 1 else 2
    cases = {"d3q27_box": (I.GridSpec(3, (512 // s, 256 // s, 256 // s), 1, [], (True, True, True)), "D3Q27", 216),
             "d2q9_tg": (I.taylor_green_spec(8192 // s, 0, 0, 1), "D2Q9", 72)}
    out = {"storage": "f32", "model": "rr", "note": "identical arithmetic (readouts bitwise equal, tests/test_gpu_aa.py)"}
    for name, (spec, lat, bpu) in cases.items():
        for mode in ("ab", "aa"):
            ctx = lt.Context(spec.dim, device=local, stream=stream.cuda_stream)
            ctx.configure(spec, lat, "rr", "f32", nu0=0.01, streaming=mode)
            ctx.use_graph(True)
            lv, xyz, _ = ctx.cells()
            n = lv.size
            rho = 1.0 + 1e-3 * I.uniform_at(71, 0, xyz[:, :spec.dim], 0)
            u = 0.02 + 1e-3 * np.stack([I.uniform_at(72 + k, 0, xyz[:, :spec.dim], 0) for k in range(spec.dim)])
            ctx.init_fields(rho, u)
            ctx.step(4)
            K = 20
            ms = _event_ms(stream, lambda: ctx.step(K)) / K
            ctx.sync()
            st = ctx.stats()
            out[f"{name}_{mode}"] = {"cells": int(n), "ms_per_step": ms, "value": n / ms / 1e3, "unit": "MLUPS",
                                     "device_gb": st.device_bytes / 1e9,
                                     "roofline": roofline(n, ms, bpu, None, None, local)}
            ctx.close()
    free, total = torch.cuda.mem_get_info(local)
    # D3Q27 FP32: 27 x 4 bytes per population buffer and cell, plus tables (~ 8 bytes per cell)
    for mode, nbuf in (("ab", 2), ("aa", 1)):
        out[f"largest_d3q27_f32_cells_{mode}"] = int(0.95 * free / (nbuf * 108 + 8))
    out["free_gb"] = free / 1e9
    return out


def form_batched(args, stream, local):
    """48 uneven 2D cases (D2Q9 Taylor-Green and D2Q37 Sod tubes, 2-4 levels): one batched
    launch per lattice group per fine iteration (CUDA graph of the schedule period) against
    stepping the cases one after another, each with its own graph."""
    from paper_2504_04465_b300 import lbmtree as lt
    cases = I.batch_cases()
    out = {"workload": "48 cases from the batch recipe (PCG64 seed 48), 23 M cells",
           "step": "16 fine iterations of every case (one period of the 4-level schedule)"}
    for storage in ("f32", "f16dev"):
        ctxs = []
        for cs in cases:
            c = lt.Context(2, device=local, stream=stream.cuda_stream)
            c.configure(cs["spec"], cs["lattice"], cs["model"], storage, **cs["params"])
            lvl, xyz, _ = c.cells()
            n = lvl.size
            rho, u, T = np.ones(n), np.zeros((2, n)), np.zeros(n)
            for L in np.unique(lvl):
                m = lvl == L
                r = cs["fields"](int(L), xyz[m, :2])
                rho[m], u[:, m] = r[0], r[1]
                if len(r) > 2:
                    T[m] = r[2]
            c.init_fields(rho, u, T if cs["model"] == "poly_ddf" else None)
            c.use_graph(True)
            ctxs.append(c)
        stats = [c.stats() for c in ctxs]
        upd = sum(s.cell_updates * 16 // (1 << (s.n_levels - 1)) for s in stats)
        coarse = [16 >> (s.n_levels - 1) for s in stats]     # 16 fine iterations in coarse steps
        b = lt.Batch(ctxs, stream.cuda_stream)
        b.use_graph(True)
        b.step_fine(32)
        reps = 4
        ms_b = _event_ms(stream, lambda: b.step_fine(16), reps)
        b.sync()
        l0 = b.info()["launches"]
        for c, k in zip(ctxs, coarse):
            c.step(k)
        ms_s = _event_ms(stream, lambda: [c.step(k) for c, k in zip(ctxs, coarse)], reps)
        for c in ctxs:
            c.sync()
        out[storage] = {"batched_ms": ms_b, "sequential_ms": ms_s, "speedup": ms_s / ms_b,
                        "value": upd / ms_b / 1e3, "unit": "MLUPS", "sequential_value": upd / ms_s / 1e3,
                        "groups": b.info()["groups"]}
        b.close()
        for c in ctxs:
            c.close()
    return out


def run_ours(args, world, rank, local):
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    spec = I.sphere_spec(args.scale)
    graph = not args.no_graph
    block = tuple(args.block) if args.block else DEFAULT_BLOCK[args.storage]
    variant = args.variant if args.variant is not None else DEFAULT_VARIANT[args.storage]
    tuned = None
    if args.autotune:
        from paper_2504_04465_b300 import autotune as AT
        log = (lambda s: print(s, file=sys.stderr, flush=True)) if rank == 0 else None
        block, variant, table = AT.tune(
            lambda shp, strm: make_context(spec, args.storage, local, strm, False, args.scale, shp),
            lambda c: c.init_fields(*host_fields(c)), AT.CANDIDATES_3D, device=local, log=log)
        tuned = {f"{k[0]}:{k[1]}": round(v, 4) for k, v in table.items()}
    ctx = make_context(spec, args.storage, local, stream.cuda_stream, graph, args.scale, block, variant)
    rho, u = host_fields(ctx)
    ctx.init_fields(rho, u)
    st = ctx.stats()
    updates_per_step = st.cell_updates              # one coarse step
    for _ in range(args.warmup):
        ctx.step(1)
    ctx.sync()
    l0 = ctx.stats().kernel_launches
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            ev0.record(stream)
            ctx.step(args.steps)
            ev1.record(stream)
        torch.cuda.synchronize()
        ctx.sync()
        if dist:
            dist.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = ctx.stats().kernel_launches - l0
    t_max, total_updates = replica_totals(ms, updates_per_step * args.steps, dist, "cuda")
    value = total_updates / (t_max * 1e-3) / 1e6
    # roofline of the step kernel: it is the only kernel of the timed region
    bpu = BYTES_PER_UPDATE[args.storage]
    achieved = bpu * updates_per_step * args.steps / (ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    traffic, tnote = counter(f"d3q27:{args.storage}", "dram")
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_kind": peak_kind, "bytes_per_update": bpu,
            "per": "coarse step: the interior and general step kernels of 8 fine iterations (event-timed together)",
            "traffic": None if traffic is None else traffic * updates_per_step, "traffic_per_update": traffic,
            "traffic_source": tnote + ("" if traffic is None else
                                       " (DRAM bytes per update at half extents, times this step's updates)")}
    # end to end through the public API with host buffers: upload the fields, step, read the
    # conserved totals every step and the moments at the end
    e2e = None
    if not args.no_e2e:
        n = rho.size
        # inputs and outputs in pinned host memory
        pin = lambda shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        h_rho, h_u = pin(n), pin((3, n))
        h_rho[:] = rho
        h_u[:] = u
        o_rho, o_u, o_T = pin(n), pin(3 * n), pin(n)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.init_fields(h_rho, h_u)
        for _ in range(args.steps):
            ctx.step(1)
            ctx.conserved()
        ctx.moments(out=(o_rho, o_u, o_T))
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        h2d = (h_rho.nbytes + h_u.nbytes) / args.steps
        d2h = 5 * 8 + (o_rho.nbytes + o_u.nbytes + o_T.nbytes) / args.steps
        e2e = {"value": updates_per_step * args.steps * world / te / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "note": "pinned host buffers; init_fields once, step + conserved() (FP64 totals read back) per "
                       "step, read_moments once; bytes per step are the totals / steps"}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu:
        cpu = cpu_baseline(args.cpu_seconds)
    forms = None
    if not args.no_forms and args.storage == "f32":
        forms = {}
        for name, fn in (("fp16_store", lambda: form_fp16(args, stream, local, t_max / args.steps)),
                         ("learned", lambda: form_learned(args, stream, local)),
                         ("batched", lambda: form_batched(args, stream, local)),
                         ("d2q37_sod", lambda: form_d2q37(args, stream, local)),
                         ("d2q9_tg", lambda: form_d2q9(args, stream, local)),
                         ("sod_numerical", lambda: form_sod_numerical(args, stream, local)),
                         ("d2q21_weak", lambda: form_d2q21_weak(args, stream, local)),
                         ("naca37", lambda: form_naca37(args, stream, local)),
                         ("riemann12", lambda: form_riemann12(args, stream, local)),
                         ("aa", lambda: form_aa(args, stream, local))):
            if name not in args.forms.split(","):
                continue
            try:
                forms[name] = fn()
            except Exception as e:                  # report, keep the main line
                forms[name] = {"error": f"{type(e).__name__}: {e}"}
    line = {"metric": "fine-equivalent MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
            "config": {"workload": WORKLOAD if args.scale == 1 else f"{WORKLOAD}, extents / {args.scale}",
                       "storage": args.storage, "cells": int(sum(st.n_cells[:4])),
                       "n_eq": st.n_eq, "cell_updates_per_step": int(updates_per_step),
                       "step": "one coarse step = 8 fine iterations", "cuda_graph": graph,
                       "block": list(block), "variant_min_blocks": ctx.variants()[variant],
                       "autotune_ms_per_step": tuned,
                       "l2": "inputs larger than L2 (9.7 GB of populations at f32)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roof, "pipe_peaks": pipe_peaks(local), "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk.summary(), "forms": forms}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16dev", "f64"])
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP16 / learned-guess / batched forms")
    ap.add_argument("--forms", default="fp16_store,learned,batched,d2q37_sod,d2q9_tg,sod_numerical,d2q21_weak,naca37,riemann12,aa",
                    help="which forms to run (comma list; sod_numerical is the paper's Sec. 7.6 Sod benchmark)")
    ap.add_argument("--sod-lattices", default="all", help="sod_numerical: lattices (D2Q21,D2Q37 or all)")
    ap.add_argument("--sod-grids", default="unif,band,sqr",
                    help="sod_numerical: grids (hori is refused: its interface meets the Neumann faces)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--block", type=int, nargs=3, default=None)
    ap.add_argument("--variant", type=int, default=None)
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--scale", type=int, default=1, choices=[1, 2, 4],
                    help="1: the full workload; 2, 4: copies with extents divided by 2, 4 (profiling, tests)")
    ap.add_argument("--counters", default=None,
                    help="run one kernel path's captured case (e.g. d3q27:f32) for an ncu capture and exit")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    world, rank, local = dist_setup()
    if args.counters:
        run_counters(args, local)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
