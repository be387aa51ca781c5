"""Build the CUDA library liblbmtree.so in-tree for sm_103a (B300).

    python -m paper_2504_04465_b300.build [-v] [-f]

Each lattice's kernels live in their own translation unit and compile in parallel.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "liblbmtree.so")
SOURCES = ["k_d2q9.cu", "k_d3q27.cu", "k_d2q37.cu", "k_d2q21.cu", "k_d2q21w.cu", "noalloc.cu", "k_mlp.cu", "k_io.cu", "api.cpp", "builder.cpp", "weights.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = os.environ.get("NVCC") or "/usr/local/cuda/bin/nvcc"
    return cand if os.path.exists(cand) else "nvcc"


def build(verbose: bool = False, force: bool = False, extra: list[str] | None = None) -> str:
    """Compile every source for sm_103a and link liblbmtree.so next to this file."""
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(HERE, "..", "include", "lbmtree.h"))
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(d) for d in deps):
        return LIB
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    objs, procs = [], []
    for s in srcs:
        o = os.path.join(objdir, os.path.basename(s) + ".o")
        cmd = [_nvcc(), "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-fopenmp",
               "-I", os.path.join(HERE, "..", "include"), "-c", s, "-o", o, *(extra or [])]
        if verbose and s.endswith(".cu"):
            cmd += ["-Xptxas", "-v"]
        procs.append((s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        objs.append(o)
    failed = False
    for s, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stdout.write(out)
        if p.returncode:
            failed = True
            sys.stdout.write(f"\n*** compile failed: {s}\n")
    if failed:
        raise RuntimeError("nvcc failed")
    cmd = [_nvcc(), "-shared", *ARCH, "-Xcompiler", "-fopenmp", "-o", LIB, *objs, "-lgomp", "-lcudart"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode:
        sys.stdout.write(r.stdout)
        raise RuntimeError("link failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
