"""Build libmegopolis.so in-tree for sm_103a with nvcc.

Each translation unit under csrc/ is compiled in parallel to an object file,
then linked into paper_2109_13504_gb300/_build/libmegopolis.so.  The CUDA
runtime is linked statically (nvcc's default), so the library needs only the
driver at run time.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmegopolis.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE,
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build")
    return path


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _inputs_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "megopolis.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


# The bounds-checked build (-DMEGO_BOUNDS_CHECK): every index the chains form
# is checked against n and a bad one is recorded in the fault word instead of
# being used.  It holds the single-resample entry points only (the C ABI's
# host code, the bound and the resample kernels) and is built on demand by
# the test that uses it, not by build().
CHECKED_SOURCES = ("capi.cu", "bound.cu", "resample_megopolis.cu", "resample_metropolis.cu",
                   "resample_c1.cu", "resample_c2.cu")
CHECKED_DIR = os.path.join(BUILD, "checked")
CHECKED_LIB = os.path.join(CHECKED_DIR, "libmegopolis_checked.so")


def _build_lib(srcs, out_dir, lib, defines, verbose, ptxas_info) -> str:
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + ["-D" + d for d in defines]

    def compile_one(src: str) -> str:
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        proc = subprocess.run(cmd, capture_output=True, text=True)
        if proc.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, proc.stderr))
        if ptxas_info and proc.stderr:
            print(proc.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    proc = subprocess.run(cmd, capture_output=True, text=True)
    if proc.returncode != 0:
        raise RuntimeError("nvcc link failed:\n%s" % proc.stderr)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _inputs_mtime():
        return LIB
    return _build_lib(sources(), BUILD, LIB, [], verbose, ptxas_info)


def build_checked(force: bool = False, verbose: bool = False) -> str:
    if (not force and os.path.exists(CHECKED_LIB)
            and os.path.getmtime(CHECKED_LIB) >= _inputs_mtime()):
        return CHECKED_LIB
    srcs = [os.path.join(CSRC, f) for f in CHECKED_SOURCES]
    return _build_lib(srcs, CHECKED_DIR, CHECKED_LIB, ["MEGO_BOUNDS_CHECK"], verbose, False)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="-v" in sys.argv))
