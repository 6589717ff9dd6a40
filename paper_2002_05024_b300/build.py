"""Build step: compile the CUDA sources of the library into
paper_2002_05024_b300/_lib/libevec.so for sm_103a (B300), in-tree, and the
checked build (-DEVEC_CHECK: bounds checks of the kernels' main device
accesses, reported as EVEC_EBOUNDS) into _lib/libevec_check.so.

Each .cu file is compiled to its own object (in parallel; a file is
recompiled when it, or any header, is newer than its object), then the
objects are linked into the shared library."""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB_DIR = os.path.join(HERE, "_lib")
OBJ_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(LIB_DIR, "libevec.so")
CHECK_LIB = os.path.join(LIB_DIR, "libevec_check.so")
CHECK_OBJ_DIR = os.path.join(HERE, "_build_check")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]
LFLAGS = ["-shared", "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(HERE, "..", "include", "*.h")))


def _obj(src, checked=False):
    return os.path.join(CHECK_OBJ_DIR if checked else OBJ_DIR, os.path.basename(src)[:-3] + ".o")


def up_to_date(checked: bool = False) -> bool:
    lib = CHECK_LIB if checked else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in sources() + headers())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build libevec.so (checked: libevec_check.so) when a source is newer."""
    lib = CHECK_LIB if checked else LIB
    obj_dir = CHECK_OBJ_DIR if checked else OBJ_DIR
    if not force and up_to_date(checked):
        return lib
    os.makedirs(LIB_DIR, exist_ok=True)
    os.makedirs(obj_dir, exist_ok=True)
    hdr_t = max((os.path.getmtime(f) for f in headers()), default=0.0)
    srcs = sources()
    stale = [s for s in srcs if force or not os.path.exists(_obj(s, checked)) or
             os.path.getmtime(_obj(s, checked)) < max(os.path.getmtime(s), hdr_t)]
    flags = CFLAGS + (["-DEVEC_CHECK"] if checked else [])

    def compile_one(src):
        out = _obj(src, checked)
        tmp = out + f".tmp{os.getpid()}"
        cmd = [NVCC, *ARCH, *flags, "-c", "-o", tmp, src]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)

    workers = max(1, min(len(stale), os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as pool:
        for f in [pool.submit(compile_one, s) for s in stale]:
            f.result()
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.run([NVCC, *ARCH, *LFLAGS, "-o", tmp, *[_obj(s, checked) for s in srcs]],
                   check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                checked="--checked" in sys.argv))
