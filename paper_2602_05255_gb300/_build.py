"""Builds the CUDA library liblrugb.so in-tree for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library next to this file.  Re-running only recompiles changed units.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblrugb.so")
LIB_DEBUG = os.path.join(HERE, "liblrugb_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
# (source, object, extra defines): the kernel file is split by dtype
UNITS = [
    ("lrugb_api.cu", "lrugb_api.o", []),
    ("lru_kernels.cu", "lru_kernels_f64.o", ["-DLRU_INST_DTYPE=double", "-DLRU_INST_PRIMARY", "-DLRU_NO_STEP"]),
    ("lru_kernels.cu", "lru_kernels_c128.o", ["-DLRU_INST_DTYPE=c128", "-DLRU_NO_STEP"]),
    ("lru_kernels.cu", "lru_kernels_f32.o", ["-DLRU_INST_DTYPE=float", "-DLRU_NO_STEP"]),
    ("lru_kernels.cu", "lru_kernels_c64.o", ["-DLRU_INST_DTYPE=c64", "-DLRU_NO_STEP"]),
    # the persistent fused step, per dtype
    ("lru_kernels.cu", "lru_step_f64.o", ["-DLRU_INST_DTYPE=double", "-DLRU_STEP_ONLY"]),
    ("lru_kernels.cu", "lru_step_c128.o", ["-DLRU_INST_DTYPE=c128", "-DLRU_STEP_ONLY"]),
    ("lru_kernels.cu", "lru_step_f32.o", ["-DLRU_INST_DTYPE=float", "-DLRU_STEP_ONLY"]),
    ("lru_kernels.cu", "lru_step_c64.o", ["-DLRU_INST_DTYPE=c64", "-DLRU_STEP_ONLY"]),
    ("refresh.cu", "refresh.o", []),
    ("refresh_oz.cu", "refresh_oz.o", []),
    ("flush_tc.cu", "flush_tc.o", []),
    ("adjoint.cu", "adjoint.o", []),
]


def _nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblrugb.so")


def _deps_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    paths.append(os.path.join(os.path.dirname(HERE), "include", "lrugb.h"))
    return max(os.path.getmtime(p) for p in paths if os.path.isfile(p))


def build(verbose: bool = False, debug: bool = False) -> str:
    """Compiles (the changed units of) liblrugb.so, or with debug=True
    liblrugb_debug.so (-DLRU_DEBUG: device-side index checks that record a
    sticky error, canary-guarded handle allocations)."""
    nvcc = _nvcc()
    bdir = os.path.join(BUILD, "debug") if debug else BUILD
    lib = LIB_DEBUG if debug else LIB
    extra = ["-DLRU_DEBUG"] if debug else []
    os.makedirs(bdir, exist_ok=True)
    dep = _deps_mtime()
    jobs = []
    objs = []
    for src_name, obj_name, defs in UNITS:
        src = os.path.join(CSRC, src_name)
        obj = os.path.join(bdir, obj_name)
        objs.append(obj)
        if not os.path.exists(obj) or os.path.getmtime(obj) < dep:
            jobs.append([nvcc, *ARCH, *FLAGS, *extra, *defs, "-c", src, "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
    for cmd, r in zip(jobs, results):
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed ({' '.join(cmd[-3:])}):\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
    if jobs or not os.path.exists(lib):
        cmd = [nvcc, *ARCH, "-shared", "-o", lib, *objs, "-cudart", "shared",
               "-Xlinker", "-rpath=/usr/local/cuda/lib64"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return lib


if __name__ == "__main__":
    import sys
    print(build(verbose=True, debug="--debug" in sys.argv))
