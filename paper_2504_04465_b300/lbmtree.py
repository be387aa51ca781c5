"""Thin Python binding of liblbmtree.so (the C ABI declared in include/lbmtree.h).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.  The
library must have been built (``python -m paper_2504_04465_b300.build``); importing this module
without it raises ImportError -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbmtree.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2504_04465_b300.build`")

_lib = C.CDLL(LIB_PATH)

# ------------------------------------------------------------------ constants (include/lbmtree.h)
OK = 0
ERR = {-1: "ARG", -2: "STATE", -3: "CUDA", -4: "OOM", -5: "GRID", -6: "NEWTON", -7: "NONFINITE",
       -10: "UNSUPPORTED"}
LATTICE = {"D2Q9": 9, "D2Q13": 13, "D2Q21": 21, "D2Q37": 37, "D3Q27": 27}
MODEL = {"bgk": 1, "rr": 2, "poly_ddf": 3, "num_ddf": 4, "trt": 5}
STORAGE = {"f64": 1, "f32": 2, "f16dev": 3}
FACE_KIND = {"periodic": 0, "dirichlet": 1, "dirichlet_rho": 2, "neumann": 3, "wall": 4}
GUESS = {"warm": 0, "zero": 1, "poly": 2, "mlp": 3}
FACES = ["x-", "x+", "y-", "y+", "z-", "z+"]
CELL_FLUID, CELL_CGHOST, CELL_FGHOST, CELL_BC, CELL_SOLID = 1, 2, 3, 4, 5


class CollisionParams(C.Structure):
    _fields_ = [("nu0", C.c_double), ("T0", C.c_double), ("gamma", C.c_double), ("sensor_on", C.c_int),
                ("sensor_A", C.c_double), ("newton_tol", C.c_double), ("newton_max_iter", C.c_int),
                ("guess", C.c_int), ("rho_ref", C.c_double), ("newton_fp32", C.c_int), ("trace_eq", C.c_int),
                ("trt_magic", C.c_double)]


class Box(C.Structure):
    _fields_ = [("level", C.c_int), ("lo", C.c_int64 * 3), ("hi", C.c_int64 * 3)]


class Shape(C.Structure):
    _fields_ = [("kind", C.c_int), ("p", C.c_double * 8)]


class Stats(C.Structure):
    _fields_ = [("n_cells", C.c_int64 * 8), ("n_blocks", C.c_int64 * 8), ("n_eq", C.c_double),
                ("n_levels", C.c_int), ("block", C.c_int * 3), ("newton_iter_sum", C.c_int64),
                ("newton_updates", C.c_int64), ("newton_nonconverged", C.c_int64),
                ("newton_hist", C.c_int64 * 16), ("fine_iterations", C.c_int64),
                ("kernel_launches", C.c_int64), ("device_bytes", C.c_int64), ("cell_updates", C.c_int64),
                ("n_general_blocks", C.c_int64 * 8)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_sig = {
    "lbm_create": [C.POINTER(_P), C.c_int, C.c_int, _P],
    "lbm_destroy": [_P],
    "lbm_set_lattice": [_P, C.c_int],
    "lbm_set_collision": [_P, C.c_int, C.POINTER(CollisionParams)],
    "lbm_set_precision": [_P, C.c_int],
    "lbm_set_sponge": [_P, _D, C.c_double, C.c_double, C.c_double, C.c_double],
    "lbm_set_streaming": [_P, C.c_int],
    "lbm_grade_level_map": [C.c_int, C.POINTER(C.c_int64), C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_uint8)],
    "lbm_amr_level_map": [_P, C.c_double, C.POINTER(C.c_uint8), C.POINTER(C.c_uint8)],
    "lbm_remesh": [_P, C.POINTER(C.c_uint8)],
    "lbm_set_boundary": [_P, C.c_int, C.c_int, _D],
    "lbm_set_block": [_P, C.c_int, C.c_int, C.c_int],
    "lbm_build_grid": [_P, C.POINTER(C.c_int64), C.c_int, C.POINTER(Box), C.c_int, C.POINTER(Shape), C.c_int],
    "lbm_build_grid_map": [_P, C.POINTER(C.c_int64), C.c_int, C.POINTER(C.c_uint8), C.POINTER(Shape), C.c_int],
    "lbm_cells": [_P, C.POINTER(C.c_int64), C.POINTER(C.POINTER(C.c_int32)), C.POINTER(C.POINTER(C.c_int32)),
                  C.POINTER(C.POINTER(C.c_uint8))],
    "lbm_velocities": [_P, C.POINTER(C.c_int), C.POINTER(C.POINTER(C.c_int32))],
    "lbm_init_fields": [_P, _D, _D, _D],
    "lbm_step": [_P, C.c_int64],
    "lbm_step_fine": [_P, C.c_int64],
    "lbm_use_graph": [_P, C.c_int],
    "lbm_sync": [_P],
    "lbm_read_moments": [_P, _D, _D, _D],
    "lbm_read_populations": [_P, C.c_int, _D],
    "lbm_conserved": [_P, _D],
    "lbm_stats": [_P, C.POINTER(Stats)],
    "lbm_variants": [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "lbm_set_variant": [_P, C.c_int],
    "lbm_conserved_noalloc": [_P, C.c_void_p],
    "lbm_mlp_forward": [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p],
    "lbm_mlp_grad": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p],
    "lbm_mlp_adam": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_float, C.c_void_p],
    "lbm_mlp_forward_tc": [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p],
    "lbm_mlp_grad_tc": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p],
    "lbm_mlp_set": [_P, C.POINTER(C.c_float), _D, _D],
    "lbm_newton_batch": [_P, C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p],
    "lbm_mlp_nparams": [],
    "lbm_mlp_get": [_P, C.POINTER(C.c_float), _D, _D],
    "lbm_set_guess": [_P, C.c_int],
    "lbm_set_allocator": [_P, C.c_void_p],
    "lbm_save": [_P, C.c_char_p],
    "lbm_load": [_P, C.c_char_p],
    "lbm_autotune": [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_float)],
    "lbm_lattice_info": [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), _D],
    "lbm_set_newton_precision": [_P, C.c_int, C.c_double],
    "lbm_batch_create": [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int, C.c_void_p],
    "lbm_batch_destroy": [C.c_void_p],
    "lbm_batch_use_graph": [C.c_void_p, C.c_int],
    "lbm_batch_step": [C.c_void_p, C.c_int64],
    "lbm_batch_sync": [C.c_void_p],
    "lbm_batch_info": [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
    "lbm_mlp_train": [_P, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p],
    "lbm_pipe_peak": [C.c_int, C.c_int, C.c_int, _D, C.POINTER(C.c_float)],
}
for _name, _args in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.lbm_last_error.argtypes = []
_lib.lbm_last_error.restype = C.c_char_p

EXPORTED = sorted(list(_sig) + ["lbm_last_error"])


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", C.c_void_p)]


def torch_allocator(device: int = 0, stream: int = 0) -> Allocator:
    """lbm_allocator backed by PyTorch's caching allocator (keep the returned object alive as
    long as the context)."""
    import torch

    def _alloc(nbytes, _user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream)
        except Exception:
            return None

    def _free(ptr, _user):
        torch.cuda.caching_allocator_delete(ptr)

    a = Allocator(_ALLOC_FN(_alloc), _FREE_FN(_free), None)
    a._keep = (_alloc, _free)
    return a


class Batch:
    """Several contexts stepped together (lbm_batch_*)."""

    def __init__(self, cases, stream: int = 0):
        self.cases = list(cases)                 # keeps the contexts alive
        arr = (C.c_void_p * len(self.cases))(*[c._h.value for c in self.cases])
        h = C.c_void_p()
        _check(_lib.lbm_batch_create(C.byref(h), arr, len(self.cases), C.c_void_p(stream)), "lbm_batch_create")
        self._h = h

    def use_graph(self, on: bool = True) -> None:
        _check(_lib.lbm_batch_use_graph(self._h, int(on)), "lbm_batch_use_graph")

    def step_fine(self, n: int) -> None:
        _check(_lib.lbm_batch_step(self._h, n), "lbm_batch_step")

    def sync(self) -> None:
        _check(_lib.lbm_batch_sync(self._h), "lbm_batch_sync")

    def info(self):
        g, l, s = C.c_int(), C.c_int64(), C.c_int64()
        _check(_lib.lbm_batch_info(self._h, C.byref(g), C.byref(l), C.byref(s)), "lbm_batch_info")
        return {"groups": g.value, "launches": l.value, "span": s.value}

    def close(self) -> None:
        if self._h:
            _lib.lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MlpTrainParams(C.Structure):
    _fields_ = [("steps", C.c_int), ("batch", C.c_int), ("lr", C.c_double), ("lr_final", C.c_double),
                ("seed", C.c_uint64), ("final_loss", C.c_float), ("tensor_cores", C.c_int)]


def lattice_info(name: str) -> dict:
    q, d, r, c2 = C.c_int(), C.c_int(), C.c_int(), C.c_double()
    _check(_lib.lbm_lattice_info(LATTICE[name], C.byref(q), C.byref(d), C.byref(r), C.byref(c2)), "lbm_lattice_info")
    return {"Q": q.value, "D": d.value, "reach": r.value, "cs2": c2.value}


def lattice_cs2(name: str) -> float:
    return lattice_info(name)["cs2"]


PIPE_KIND = {"fp32": 0, "fp64": 1, "fp32x2": 2}


def grade_level_map(level_map, n_levels: int, lattice: str, periodic) -> np.ndarray:
    """The library's grading of a level map (array of shape extent), returned as a new array."""
    m = np.asarray(level_map, dtype=np.uint8)
    ext = (C.c_int64 * 3)(*(list(m.shape) + [1, 1, 1])[:3])
    per = (C.c_int * 3)(*(list(int(bool(p)) for p in periodic) + [1, 1, 1])[:3])
    flat = np.ascontiguousarray(m.ravel(order="F"))
    _check(_lib.lbm_grade_level_map(m.ndim, ext, n_levels, LATTICE[lattice], per, flat.ctypes.data_as(C.POINTER(C.c_uint8))),
           "lbm_grade_level_map")
    return flat.reshape(m.shape, order="F")


def pipe_peak(kind: str, device: int = 0, iters: int = 8192) -> tuple[float, float]:
    """(flop/s, ms) of a fused multiply-add pipe of ``device`` (lbm_pipe_peak): "fp32", "fp64"
    or "fp32x2" (packed FP32 pairs)."""
    out, ms = C.c_double(), C.c_float()
    _check(_lib.lbm_pipe_peak(device, PIPE_KIND[kind], iters, C.byref(out), C.byref(ms)), "lbm_pipe_peak")
    return out.value, ms.value


def mlp_nparams() -> int:
    return _lib.lbm_mlp_nparams()


def mlp_forward(d_params: int, d_x: int, n: int, d_y: int, stream: int = 0, tensor_cores: bool = False) -> None:
    f = _lib.lbm_mlp_forward_tc if tensor_cores else _lib.lbm_mlp_forward
    _check(f(C.c_void_p(d_params), C.c_void_p(d_x), n, C.c_void_p(d_y), C.c_void_p(stream)), "lbm_mlp_forward")


def mlp_grad(d_params: int, d_x: int, d_t: int, n: int, d_grad: int, d_loss: int, stream: int = 0,
             tensor_cores: bool = False) -> None:
    f = _lib.lbm_mlp_grad_tc if tensor_cores else _lib.lbm_mlp_grad
    _check(f(C.c_void_p(d_params), C.c_void_p(d_x), C.c_void_p(d_t), n, C.c_void_p(d_grad), C.c_void_p(d_loss),
             C.c_void_p(stream)), "lbm_mlp_grad")


def mlp_adam(d_params: int, d_grad: int, d_m: int, d_v: int, step: int, lr: float, stream: int = 0) -> None:
    _check(_lib.lbm_mlp_adam(C.c_void_p(d_params), C.c_void_p(d_grad), C.c_void_p(d_m), C.c_void_p(d_v), step,
                             C.c_float(lr), C.c_void_p(stream)), "lbm_mlp_adam")


class LbmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib.lbm_last_error().decode(errors="replace")
        super().__init__(f"{where}: {ERR.get(code, code)} ({msg})")


def _check(code: int, where: str) -> None:
    if code != OK:
        raise LbmError(code, where)


def _dptr(a: np.ndarray | None):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


class Context:
    """One simulation: a grid, its populations and its stream (see include/lbmtree.h)."""

    def __init__(self, dim: int, device: int = 0, stream: int | None = None):
        h = _P()
        _check(_lib.lbm_create(C.byref(h), dim, device, _P(stream) if stream else None), "lbm_create")
        self._h = h
        self.dim = dim

    def close(self) -> None:
        if getattr(self, "_h", None):
            _lib.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -------------------------------------------------------------- configuration
    def set_lattice(self, name: str) -> None:
        _check(_lib.lbm_set_lattice(self._h, LATTICE[name]), "lbm_set_lattice")

    def set_collision(self, model: str, nu0: float = 0.0, T0: float = 0.0, gamma: float = 1.4,
                      sensor_A: float | None = None, newton_tol: float = 0.0, newton_max_iter: int = 50,
                      guess: str = "warm", rho_ref: float = 1.0, newton_fp32: bool = False,
                      trace_eq: bool = False, trt_magic: float = 0.25) -> None:
        p = CollisionParams(nu0, T0, gamma, int(sensor_A is not None), sensor_A or 0.0, newton_tol,
                            newton_max_iter, GUESS[guess], rho_ref, int(newton_fp32), int(trace_eq), trt_magic)
        _check(_lib.lbm_set_collision(self._h, MODEL[model], C.byref(p)), "lbm_set_collision")

    def set_streaming(self, mode: str) -> None:
        """'ab' (two buffers, the default) or 'aa' (one buffer updated in place); before the build."""
        _check(_lib.lbm_set_streaming(self._h, {"ab": 0, "aa": 1}[mode]), "lbm_set_streaming")

    def set_sponge(self, centre, r0: float, r1: float, sigma_max: float, rho_inf: float = 1.0) -> None:
        """Far-field relaxation (Eq. relaxation_pressure), finest units; sigma_max = 0 switches it off."""
        c = np.zeros(3)
        c[: len(centre)] = centre
        _check(_lib.lbm_set_sponge(self._h, _dptr(c), r0, r1, sigma_max, rho_inf), "lbm_set_sponge")

    def save(self, path: str) -> None:
        _check(_lib.lbm_save(self._h, str(path).encode()), "lbm_save")

    def load(self, path: str) -> None:
        _check(_lib.lbm_load(self._h, str(path).encode()), "lbm_load")

    def autotune(self, n_coarse: int = 4):
        """Select the fastest step variant; returns (variant, ms per coarse step of each)."""
        nv = len(self.variants())
        best = C.c_int()
        ms = (C.c_float * nv)()
        _check(_lib.lbm_autotune(self._h, n_coarse, C.byref(best), ms), "lbm_autotune")
        return best.value, list(ms)

    def set_allocator(self, allocator: "Allocator | None") -> None:
        """Device memory of the grid from ``allocator`` (see torch_allocator); None: cudaMalloc."""
        self._allocator = allocator
        _check(_lib.lbm_set_allocator(self._h, C.byref(allocator) if allocator is not None else None),
               "lbm_set_allocator")

    def set_guess(self, guess: str) -> None:
        _check(_lib.lbm_set_guess(self._h, GUESS[guess]), "lbm_set_guess")

    def set_newton_precision(self, fp32: bool, tol: float = 0.0) -> None:
        _check(_lib.lbm_set_newton_precision(self._h, int(fp32), tol), "lbm_set_newton_precision")

    def set_precision(self, storage: str) -> None:
        _check(_lib.lbm_set_precision(self._h, STORAGE[storage]), "lbm_set_precision")

    def set_boundary(self, face: str, kind: str, rho: float = 1.0, u=(0.0, 0.0, 0.0), T: float = 0.0) -> None:
        v = np.array([rho, *(list(u) + [0.0] * 3)[:3], T], dtype=np.float64)
        _check(_lib.lbm_set_boundary(self._h, FACES.index(face), FACE_KIND[kind], _dptr(v)), "lbm_set_boundary")

    def set_block(self, bx: int, by: int, bz: int = 1) -> None:
        _check(_lib.lbm_set_block(self._h, bx, by, bz), "lbm_set_block")

    @staticmethod
    def _shapes(solids):
        sh = (Shape * max(1, len(solids)))()
        for k, s in enumerate(solids):
            if s["kind"] == "sphere":
                sh[k].kind = 1
                p = list(s["center"]) + [0.0] * (3 - len(s["center"])) + [s["radius"]]
            elif s["kind"] == "naca":
                sh[k].kind = 2
                p = [s["chord"], s["x0"], s["y0"], s.get("t", 0.12)]
            else:
                raise ValueError(s["kind"])
            sh[k].p[: len(p)] = p
        return sh

    def build_grid_map(self, extent, n_levels: int, level_map, solids=()) -> None:
        """Build from a level map (array of shape extent: the finest level wanted per finest cell)."""
        ext = (C.c_int64 * 3)(*(list(extent) + [1, 1, 1])[:3])
        self._extent = tuple(int(e) for e in extent)
        m = np.ascontiguousarray(np.asarray(level_map, dtype=np.uint8).ravel(order="F"))
        _check(_lib.lbm_build_grid_map(self._h, ext, n_levels, m.ctypes.data_as(C.POINTER(C.c_uint8)),
                                       self._shapes(solids), len(solids)), "lbm_build_grid_map")

    def amr_level_map(self, threshold: float, fixed_map=None) -> np.ndarray:
        """Graded level map (array of shape extent) from the kinetic sensor: finest level where eps
        exceeds threshold, fixed_map (or the coarsest level) elsewhere."""
        ext = self._extent
        n = int(np.prod(ext))
        out = np.zeros(n, dtype=np.uint8)
        fx = None
        if fixed_map is not None:
            fx = np.ascontiguousarray(np.asarray(fixed_map, dtype=np.uint8).ravel(order="F"))
        _check(_lib.lbm_amr_level_map(self._h, threshold, fx.ctypes.data_as(C.POINTER(C.c_uint8)) if fx is not None else None,
                                      out.ctypes.data_as(C.POINTER(C.c_uint8))), "lbm_amr_level_map")
        return out.reshape(ext, order="F")

    def remesh(self, level_map) -> None:
        """Rebuild the grid from a level map and carry the state over (coalescence / explosion)."""
        m = np.ascontiguousarray(np.asarray(level_map, dtype=np.uint8).ravel(order="F"))
        _check(_lib.lbm_remesh(self._h, m.ctypes.data_as(C.POINTER(C.c_uint8))), "lbm_remesh")

    def build_grid(self, extent, n_levels: int, boxes=(), solids=()) -> None:
        ext = (C.c_int64 * 3)(*(list(extent) + [1, 1, 1])[:3])
        self._extent = tuple(int(e) for e in extent)
        bx = (Box * max(1, len(boxes)))()
        for k, (lv, lo, hi) in enumerate(boxes):
            bx[k].level = lv
            bx[k].lo[:] = (list(lo) + [0, 0, 0])[:3]
            bx[k].hi[:] = (list(hi) + [1, 1, 1])[:3]
        sh = (Shape * max(1, len(solids)))()
        for k, s in enumerate(solids):
            if s["kind"] == "sphere":
                sh[k].kind = 1
                p = list(s["center"]) + [0.0] * (3 - len(s["center"])) + [s["radius"]]
            elif s["kind"] == "naca":
                sh[k].kind = 2
                p = [s["chord"], s["x0"], s["y0"], s.get("t", 0.12)]
            else:
                raise ValueError(s["kind"])
            sh[k].p[: len(p)] = p
        _check(_lib.lbm_build_grid(self._h, ext, n_levels, bx, len(boxes), sh, len(solids)), "lbm_build_grid")

    def configure(self, spec, lattice: str, model: str, storage: str = "f64", block=None, **coll) -> None:
        """Apply a grid specification (see paper_2504_04465_b300.inputs.GridSpec) and build."""
        self.set_lattice(lattice)
        sponge = coll.pop("sponge", None)
        streaming = coll.pop("streaming", None)
        if streaming is not None:
            self.set_streaming(streaming)
        self.set_collision(model, **coll)
        if sponge is not None:
            self.set_sponge(sponge["centre"], sponge["r0"], sponge["r1"], sponge["sigma_max"], sponge["rho_inf"])
        self.set_precision(storage)
        for ax in range(spec.dim):
            for side in "-+":
                f = "xyz"[ax] + side
                if spec.periodic[ax]:
                    self.set_boundary(f, "periodic")
                else:
                    fs = spec.faces[f]
                    kind = fs[0]
                    rho = fs[1] if len(fs) > 1 else 1.0
                    u = fs[2] if len(fs) > 2 else (0.0, 0.0, 0.0)
                    T = fs[3] if len(fs) > 3 and fs[3] is not None else 0.0
                    self.set_boundary(f, kind, rho, u, T)
        if block is not None:
            self.set_block(*block)
        if getattr(spec, "level_map", None) is not None:
            self.build_grid_map(spec.extent, spec.n_levels, spec.level_map, spec.solids)
        else:
            self.build_grid(spec.extent, spec.n_levels, spec.boxes, spec.solids)

    # -------------------------------------------------------------- cells
    def n_cells(self) -> int:
        """Number of listed cells (the length of the arrays of cells(), moments(), populations())."""
        n = C.c_int64()
        lv = C.POINTER(C.c_int32)()
        xyz = C.POINTER(C.c_int32)()
        ty = C.POINTER(C.c_uint8)()
        _check(_lib.lbm_cells(self._h, C.byref(n), C.byref(lv), C.byref(xyz), C.byref(ty)), "lbm_cells")
        return n.value

    def cells(self):
        """(level (n,), xyz (n, 3), type (n,)) in the library's cell order (copies)."""
        n = C.c_int64()
        lv = C.POINTER(C.c_int32)()
        xyz = C.POINTER(C.c_int32)()
        ty = C.POINTER(C.c_uint8)()
        _check(_lib.lbm_cells(self._h, C.byref(n), C.byref(lv), C.byref(xyz), C.byref(ty)), "lbm_cells")
        N = n.value
        return (np.ctypeslib.as_array(lv, (N,)).copy() if N else np.zeros(0, np.int32),
                np.ctypeslib.as_array(xyz, (N, 3)).copy() if N else np.zeros((0, 3), np.int32),
                np.ctypeslib.as_array(ty, (N,)).copy() if N else np.zeros(0, np.uint8))

    def velocities(self) -> np.ndarray:
        q = C.c_int()
        xi = C.POINTER(C.c_int32)()
        _check(_lib.lbm_velocities(self._h, C.byref(q), C.byref(xi)), "lbm_velocities")
        return np.ctypeslib.as_array(xi, (q.value, 3)).copy()

    # -------------------------------------------------------------- fields and stepping
    def init_fields(self, rho, u, T=None) -> None:
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        T = None if T is None else np.ascontiguousarray(T, dtype=np.float64)
        _check(_lib.lbm_init_fields(self._h, _dptr(rho), _dptr(u), _dptr(T)), "lbm_init_fields")

    def step(self, n_coarse: int) -> None:
        _check(_lib.lbm_step(self._h, n_coarse), "lbm_step")

    def step_fine(self, n_fine: int) -> None:
        _check(_lib.lbm_step_fine(self._h, n_fine), "lbm_step_fine")

    def variants(self) -> list[int]:
        """Occupancy targets of the compiled step-kernel variants (0 = model default; 100 + target:
        the interior blocks gathered directly instead of staged through shared memory)."""
        n = C.c_int()
        mb = (C.c_int * 8)()
        _check(_lib.lbm_variants(self._h, C.byref(n), mb), "lbm_variants")
        return list(mb[: n.value])

    def set_variant(self, v: int) -> None:
        _check(_lib.lbm_set_variant(self._h, v), "lbm_set_variant")

    def use_graph(self, on: bool = True) -> None:
        _check(_lib.lbm_use_graph(self._h, int(on)), "lbm_use_graph")

    def sync(self) -> None:
        _check(_lib.lbm_sync(self._h), "lbm_sync")

    # -------------------------------------------------------------- outputs
    def moments(self, out=None):
        """(rho, u (dim, n), T) in lbm_cells order; ``out`` = preallocated (rho, u, T) float64
        arrays (for instance in pinned host memory) to write into."""
        n = self.n_cells()
        if out is None:
            rho, u, T = np.empty(n), np.empty(self.dim * n), np.empty(n)
        else:
            rho, u, T = out
            if rho.size != n or u.size != self.dim * n or T.size != n:
                raise ValueError("output arrays of the wrong size")
        _check(_lib.lbm_read_moments(self._h, _dptr(rho), _dptr(u), _dptr(T)), "lbm_read_moments")
        return rho, u.reshape(self.dim, n), T

    def populations(self, which: str = "f") -> np.ndarray:
        n = self.n_cells()
        k = {"f": 0, "g": 1, "lambda": 2}[which]
        m = 8 if which == "lambda" else self.velocities().shape[0]
        out = np.empty(m * n)
        _check(_lib.lbm_read_populations(self._h, k, _dptr(out)), "lbm_read_populations")
        return out.reshape(m, n)

    def conserved(self) -> np.ndarray:
        out = np.empty(5)
        _check(_lib.lbm_conserved(self._h, _dptr(out)), "lbm_conserved")
        return out

    def conserved_noalloc(self, d_out: int) -> None:
        """Conserved totals into the caller's device buffer of 5 doubles (address d_out),
        without any device allocation in the call; asynchronous on the context's stream."""
        _check(_lib.lbm_conserved_noalloc(self._h, C.c_void_p(d_out)), "lbm_conserved_noalloc")

    def mlp_set(self, params: np.ndarray, m: np.ndarray, s: np.ndarray) -> None:
        p = np.ascontiguousarray(params, dtype=np.float32)
        m = np.ascontiguousarray(m, dtype=np.float64)
        s = np.ascontiguousarray(s, dtype=np.float64)
        _check(_lib.lbm_mlp_set(self._h, p.ctypes.data_as(C.POINTER(C.c_float)), _dptr(m), _dptr(s)), "lbm_mlp_set")

    def mlp_get(self):
        p = np.zeros(mlp_nparams(), np.float32)
        m = np.zeros(8)
        s = np.zeros(8)
        _check(_lib.lbm_mlp_get(self._h, p.ctypes.data_as(C.POINTER(C.c_float)), _dptr(m), _dptr(s)), "lbm_mlp_get")
        return p, m, s

    def mlp_train(self, d_uT: int, d_lambda: int, n: int, steps: int = 3000, batch: int = 1024, lr: float = 3e-3,
                  lr_final: float = 3e-4, seed: int = 1504, tensor_cores: bool = False) -> float:
        """Train the context's Newton-guess network; returns the final loss over the n samples."""
        p = MlpTrainParams(steps, batch, lr, lr_final, seed, 0.0, int(tensor_cores))
        _check(_lib.lbm_mlp_train(self._h, C.c_void_p(d_uT), C.c_void_p(d_lambda), n, C.byref(p)), "lbm_mlp_train")
        return float(p.final_loss)

    def newton_batch(self, d_uT: int, n: int, guess: str, d_lambda: int, d_iters: int) -> None:
        _check(_lib.lbm_newton_batch(self._h, C.c_void_p(d_uT), n, GUESS[guess], C.c_void_p(d_lambda),
                                     C.c_void_p(d_iters)), "lbm_newton_batch")

    def stats(self) -> Stats:
        s = Stats()
        _check(_lib.lbm_stats(self._h, C.byref(s)), "lbm_stats")
        return s
