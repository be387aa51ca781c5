"""Build the CUDA library liblbmtree.so in-tree for sm_103a (B300).

    python -m paper_2504_04465_b300.build [-v] [-f]

Each translation unit compiles in parallel into ``_build/``; nvcc writes a dependency file
beside each object, and an object is rebuilt only when its source, a header it includes or the
compiler flags changed (``-f`` rebuilds everything).  The heavy kernel sets (the Newton-solved
equilibria in each storage format) live in translation units of their own so that they compile
side by side.
"""
from __future__ import annotations

import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "liblbmtree.so")
OBJDIR = os.path.join(HERE, "_build")
# longest compiles first, so that they start first
SOURCES = [
    "k_d2q37_n32_f32.cu", "k_d2q37_n32_f16.cu", "k_d2q37_n32_f64.cu", "k_d2q37_n64.cu",
    "k_d2q21_n32_f32.cu", "k_d2q21_n32_f16.cu", "k_d2q21_n32_f64.cu", "k_d2q21.cu",
    "k_d2q37.cu", "k_d2q13.cu", "k_d3q27.cu", "k_d2q9.cu", "k_d2q21w.cu",
    "noalloc.cu", "k_peak.cu", "k_mlp.cu", "k_io.cu", "api.cpp", "builder.cpp", "weights.cpp",
]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = os.environ.get("NVCC") or "/usr/local/cuda/bin/nvcc"
    return cand if os.path.exists(cand) else "nvcc"


def _flags(extra) -> list[str]:
    return ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-fopenmp",
            "-I", os.path.join(HERE, "..", "include"), *(extra or [])]


def _deps(dfile: str) -> list[str] | None:
    """Prerequisites listed in an nvcc -MF dependency file (None if it is missing)."""
    try:
        with open(dfile) as fh:
            text = fh.read().replace("\\\n", " ")
    except OSError:
        return None
    _, _, rest = text.partition(":")
    return rest.split()


def _stale(src: str, obj: str, dfile: str, stamp: str, sig: str) -> bool:
    if not os.path.exists(obj):
        return True
    try:
        with open(stamp) as fh:
            if fh.read() != sig:
                return True
    except OSError:
        return True
    deps = _deps(dfile)
    if deps is None:
        return True
    t = os.path.getmtime(obj)
    for d in [src, *deps]:
        if not os.path.exists(d) or os.path.getmtime(d) > t:
            return True
    return False


def _lib_current() -> bool:
    """The library exists and is newer than every source and header (no object files needed)."""
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp", ".h", ".cuh"))]
    files.append(os.path.join(HERE, "..", "include", "lbmtree.h"))
    return all(os.path.getmtime(f) <= t for f in files)


def build(verbose: bool = False, force: bool = False, extra: list[str] | None = None) -> str:
    """Compile the stale translation units for sm_103a and link liblbmtree.so next to this file."""
    if not force and not extra and _lib_current():
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    flags = _flags(extra)
    sig = hashlib.sha256(" ".join([_nvcc(), *flags]).encode()).hexdigest()
    objs, procs = [], []
    for name in SOURCES:
        src = os.path.join(CSRC, name)
        obj = os.path.join(OBJDIR, name + ".o")
        dfile, stamp = obj[:-2] + ".d", obj[:-2] + ".flags"
        objs.append(obj)
        if not force and not _stale(src, obj, dfile, stamp, sig):
            continue
        cmd = [_nvcc(), *flags, "-MD", "-MF", dfile, "-c", src, "-o", obj]
        if verbose and name.endswith(".cu"):
            cmd += ["-Xptxas", "-v"]
        procs.append((name, stamp, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = False
    for name, stamp, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stdout.write(out)
        if p.returncode:
            failed = True
            sys.stdout.write(f"\n*** compile failed: {name}\n")
        else:
            with open(stamp, "w") as fh:
                fh.write(sig)
    if failed:
        raise RuntimeError("nvcc failed")
    if not procs and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(o) for o in objs):
        return LIB
    cmd = [_nvcc(), "-shared", *ARCH, "-Xcompiler", "-fopenmp", "-o", LIB, *objs, "-lgomp", "-lcudart"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode:
        sys.stdout.write(r.stdout)
        raise RuntimeError("link failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
