"""Builds the CUDA library ``_build/libsegmg.so`` for sm_103a (GB300) with nvcc.

Each translation unit is compiled in parallel, then linked into one shared library that
exports the C ABI of include/segmg.h.  Runs without a GPU (nvcc cross-compiles).
``build(debug=True)`` builds the bounds-checked variant ``_build/libsegmg_debug.so``
(-DMG_DEBUG: out-of-range indices of the checked accesses are skipped and recorded in device
error words that mg_debug_status reads) from its own objects under ``_build/debug``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsegmg.so")
LIB_DEBUG = os.path.join(OUT_DIR, "libsegmg_debug.so")
SOURCES = ["host.cu", "smooth_kernels.cu", "cycle_kernels.cu", "setup_kernels.cu", "bottom_kernel.cu", "sweep_tma.cu", "snapshot_tma.cu", "residual_tma.cu", "line_smoothers.cu", "aos_kernels.cu", "learned.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False, debug: bool = False) -> str:
    obj_dir = os.path.join(OUT_DIR, "debug") if debug else OUT_DIR
    lib_path = LIB_DEBUG if debug else LIB
    os.makedirs(obj_dir, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "segmg.h"))
    nvcc = _nvcc()
    common = ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-O2",
              "-I", os.path.join(ROOT, "include")]
    if ptxas_v:
        common += ["-Xptxas", "-v"]
    if debug:
        common += ["-DMG_DEBUG"]

    def compile_one(src):
        s = os.path.join(CSRC, src)
        o = os.path.join(obj_dir, src.replace(".cu", ".o"))
        if force or _stale(o, [s, *headers]):
            cmd = [nvcc, *common, "-c", s, "-o", o + ".tmp"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
            os.replace(o + ".tmp", o)
            if verbose or ptxas_v:
                sys.stderr.write(r.stderr)
        return o

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    if force or _stale(lib_path, objs):
        tmp = lib_path + f".{os.getpid()}.tmp"
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv, debug="--debug" in sys.argv))
