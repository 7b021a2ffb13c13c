"""Build libdgsem.so in-tree for sm_103a with nvcc (no cmake).

The rhs kernels are templates over (arithmetic type, dimension, degree,
volume flux); each (type, dimension) pair is its own translation unit so the
units compile in parallel.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(HERE, "libdgsem.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]

UNITS = [("dg_api.cu", [], "dg_api.o"), ("dg_noalloc.cu", [], "dg_noalloc.o"),
         ("dg_probe.cu", [], "dg_probe.o"),
         ("dg_curved.cu", [], "dg_curved.o"),
         ("dg_mhd.cu", [], "dg_mhd.o"),
         ("dg_ensemble.cu", [], "dg_ensemble.o")] + [
    ("dg_rhs_inst.cu", [f"-DDG_INST_REAL={r}", f"-DDG_INST_DIM={d}"], f"dg_rhs_{r}_{d}.o")
    for r in ("double", "float") for d in (3, 2)
] + [
    ("dg_vjp_inst.cu", [f"-DDG_INST_REAL={r}", f"-DDG_INST_DIM={d}"], f"dg_vjp_{r}_{d}.o")
    for r in ("double", "float") for d in (3, 2)
]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _sources_mtime():
    ts = [os.path.getmtime(os.path.join(CSRC, f)) for f in os.listdir(CSRC)]
    ts += [os.path.getmtime(os.path.join(INCLUDE, f)) for f in os.listdir(INCLUDE)]
    ts.append(os.path.getmtime(__file__))
    return max(ts)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= _sources_mtime():
        return SO
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_unit(unit):
        src, defs, obj = unit
        cmd = [nvcc, *ARCH, *FLAGS, *extra_flags, *defs, "-c", os.path.join(CSRC, src), "-o",
               os.path.join(BUILD, obj)]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src} {defs}:\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        for msg in ex.map(compile_unit, UNITS):
            if verbose and msg:
                print(msg)
    tmp = SO + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp,
           *[os.path.join(BUILD, u[2]) for u in UNITS],
           "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
