"""Builds the GB300 MSM library (libmsm_gb300.so) in-tree with nvcc for sm_103a.

Each CUDA translation unit is compiled in parallel, then linked into one
shared library under ``paper_2510_05961_gb300/lib``. No cmake, no torch
extension machinery: the library has a plain C ABI (include/msm_gb300.h).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "lib", "obj")
LIB = os.path.join(HERE, "lib", "libmsm_gb300.so")
# debug build with device-side index checks (-DMSM_CHECKS=1): a failed check
# sets MSM_DEV_CHECK in the status word and skips the access
OBJ_CHECKS = os.path.join(HERE, "lib", "obj_checks")
LIB_CHECKS = os.path.join(HERE, "lib", "libmsm_gb300_checks.so")
SOURCES = ["msm_api.cu", "msm_plan.cu", "k_bin.cu", "k_short.cu", "k_short_cl.cu", "k_fft.cu", "k_interp.cu", "k_grid.cu", "k_stencil.cu",
           "k_final.cu", "k_cell.cu", "msm_static.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags():
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")] + ARCH


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "msm_gb300.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=(), checks: bool = False) -> str:
    """Compile (if stale or forced) and return the path of the shared library
    (checks=True: the debug build with device-side index checks, a separate file)."""
    lib, objdir = (LIB_CHECKS, OBJ_CHECKS) if checks else (LIB, OBJ)
    extra = tuple(extra) + (("-DMSM_CHECKS=1",) if checks else ())
    if not force and not _stale(lib):
        return lib
    os.makedirs(objdir, exist_ok=True)
    cc = nvcc()

    def one(src):
        obj = os.path.join(objdir, src + ".o")
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags() + list(extra)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(one, SOURCES))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, checks="--checks" in sys.argv))
