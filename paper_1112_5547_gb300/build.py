"""Build liblbm_sc.so and libpfm.so in-tree with nvcc for sm_103a (GB300).

Each .cu file under csrc/ compiles to an object in parallel; the objects link
into a shared library with the CUDA runtime linked statically, so the library
exports only the C ABI of include/lbm_sc.h and needs no torch at link time.
csrc_pfm/ (the phase-field solver, include/pfm.h) links the same way into
libpfm.so, which also links cuFFT.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys
import time

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "liblbm_sc.so")
PFM_CSRC = os.path.join(PKG, "csrc_pfm")
PFM_LIB = os.path.join(PKG, "libpfm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm_sc.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + sorted(glob.glob(os.path.join(CSRC, "*.h")))
            + [os.path.join(ROOT, "include", "lbm_sc.h")])


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(PFM_LIB):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(PFM_LIB))
    deps = _deps() + sorted(glob.glob(os.path.join(PFM_CSRC, "*.cu"))) + [os.path.join(ROOT, "include", "pfm.h")]
    return all(os.path.getmtime(d) <= t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    """Compile csrc/*.cu for sm_103a and link liblbm_sc.so next to this file."""
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    flags = NVCC_FLAGS + ARCH + list(extra_flags or [])

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    # the library is stamped with the time the build started, so a source
    # edited while it compiles is newer and triggers the next build
    t_start = time.time()
    srcs = _sources()
    pfm_srcs = sorted(glob.glob(os.path.join(PFM_CSRC, "*.cu")))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs) + len(pfm_srcs), os.cpu_count() or 1))) as ex:
        futs = [ex.submit(compile_one, s) for s in srcs + pfm_srcs]
        objs = [f.result() for f in futs]
    for lib, lib_objs, extra in ((LIB, objs[:len(srcs)], []), (PFM_LIB, objs[len(srcs):], ["-lcufft"])):
        tmp = lib + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-cudart", "static", "-o", tmp, *lib_objs, *extra]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib)
        os.utime(lib, (t_start, t_start))
    return LIB


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
