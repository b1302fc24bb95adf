"""Build libmsc (the CUDA library behind include/msc.h) in-tree for sm_103a.

Output: paper_2409_17346_gb300/_build/libmsc.so.  The CUDA runtime is linked statically
so the library loads on any machine with the driver; nothing else is required.
"""
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC_DIR = os.path.join(HERE, "csrc")
SOURCES = [os.path.join(SRC_DIR, "msc_lib.cu"), os.path.join(SRC_DIR, "msc_server.cpp"),
           os.path.join(SRC_DIR, "msc_coder.cpp")]
DEPS = SOURCES + [os.path.join(SRC_DIR, f) for f in ("msc_cells.cuh", "msc_core.cuh", "msc_dense.cuh", "msc_runtime.h")] + \
    [os.path.join(ROOT, "include", "msc.h")]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmsc.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc_path():
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmsc")


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libmsc.so unless it is newer than every source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in DEPS):
            return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [nvcc_path(), "-std=c++17", "--expt-relaxed-constexpr", ARCH, "-O3", "-lineinfo",
           "-Xcompiler", "-fPIC", "-shared", "-o", tmp] + SOURCES + ["-ldl"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
