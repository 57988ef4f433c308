"""Compiles the CUDA library (csrc/*.cu) into lib/libdqmc_gb300.so for sm_103a.

One nvcc invocation per translation unit, run in parallel, then one link.
The result is an in-tree shared library with a plain C ABI (include/dqmc.h);
no PyTorch headers or types are involved.  The debug variant
(lib/libdqmc_gb300_debug.so) is the same sources with -DDQMC_DEBUG, whose
kernels check their index invariants on the device (include/dqmc.h).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJDIR = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIBNAME = "libdqmc_gb300.so"
DEBUG_LIBNAME = "libdqmc_gb300_debug.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def lib_path(debug: bool = False) -> str:
    return os.path.join(LIBDIR, DEBUG_LIBNAME if debug else LIBNAME)


def _nvcc() -> str:
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build the library")
    return nvcc


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h")) + [os.path.abspath(__file__)]


def up_to_date(debug: bool = False) -> bool:
    out = lib_path(debug)
    if not os.path.exists(out):
        return False
    t = os.path.getmtime(out)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, jobs: int | None = None,
          debug: bool | None = None) -> str:
    """Builds (if needed) and returns the path of the shared library.

    debug=None builds both variants (in one pool of compile jobs) and returns
    the release path; True or False builds only that variant."""
    variants = [False, True] if debug is None else [bool(debug)]
    todo = [v for v in variants if force or not up_to_date(v)]
    if not todo:
        return lib_path(variants[0])
    nvcc = _nvcc()
    os.makedirs(LIBDIR, exist_ok=True)
    srcs = _sources()

    def objdir(v):
        return OBJDIR + ("_debug" if v else "")

    def compile_one(job):
        v, src = job
        obj = os.path.join(objdir(v), os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *(["-DDQMC_DEBUG=1"] if v else []),
               "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    for v in todo:
        os.makedirs(objdir(v), exist_ok=True)
    jobs_list = [(v, src) for v in todo for src in srcs]
    with cf.ThreadPoolExecutor(max_workers=jobs or min(16, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, jobs_list))
    for v in todo:
        mine = [o for (vv, _), o in zip(jobs_list, objs) if vv == v]
        tmp = lib_path(v) + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *mine]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib_path(v))
    return lib_path(variants[0])


if __name__ == "__main__":
    print(build(force=True, verbose=True))
