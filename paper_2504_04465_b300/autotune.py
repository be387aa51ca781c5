"""Autotuner of the block shape and step-kernel variant for a given workload.

For every candidate block shape the grid is built and initialised on the device, then each
compiled variant of the step kernels (occupancy targets, see lbm_variants) is timed over a few
coarse steps with CUDA events; the fastest (shape, variant) is returned and can be cached in a
JSON file keyed by the workload name.  Tuning runs outside any timed region.
"""
from __future__ import annotations

import json
import os
import time

CANDIDATES_3D = [(8, 4, 4), (16, 4, 2), (8, 8, 2)]
CANDIDATES_2D = [(16, 16, 1), (32, 8, 1)]


def _time_variant(ctx, stream, steps: int) -> float:
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ctx.step(4)                     # builds and instantiates the graph outside the timed region
    ctx.sync()
    with torch.cuda.stream(stream):
        ev0.record(stream)
        ctx.step(steps)
        ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / steps


def tune(make_context, init, shapes, steps: int = 4, device: int = 0, log=None):
    """make_context(block, stream) -> built Context; init(ctx) initialises its fields.

    Returns (best_block, best_variant, table) with table[(block, variant)] = ms per coarse step.
    """
    import torch
    torch.cuda.set_device(device)
    stream = torch.cuda.Stream()
    table = {}
    best = None
    for shape in shapes:
        t0 = time.perf_counter()
        try:
            ctx = make_context(shape, stream.cuda_stream)
        except Exception as e:                       # shape not compiled for this lattice
            if log:
                log(f"skip {shape}: {e}")
            continue
        init(ctx)
        ctx.use_graph(True)
        for v, minb in enumerate(ctx.variants()):
            ctx.set_variant(v)
            ms = _time_variant(ctx, stream, steps)
            table[(shape, v)] = ms
            if log:
                log(f"block {shape} variant {v} (min blocks {minb}): {ms:.3f} ms/step")
            if best is None or ms < best[2]:
                best = (shape, v, ms)
        ctx.close()
        torch.cuda.synchronize()
        if log:
            log(f"  shape {shape} tuned in {time.perf_counter() - t0:.1f} s")
    if best is None:
        raise RuntimeError("no candidate could be built")
    return best[0], best[1], table


def load_cache(path: str, key: str):
    try:
        with open(path) as f:
            v = json.load(f)[key]
        return tuple(v["block"]), int(v["variant"])
    except Exception:
        return None


def save_cache(path: str, key: str, block, variant: int, ms: float) -> None:
    data = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                data = json.load(f)
        except Exception:
            data = {}
    data[key] = {"block": list(block), "variant": int(variant), "ms_per_step": ms}
    with open(path, "w") as f:
        json.dump(data, f, indent=1)
