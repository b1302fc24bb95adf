"""Compile the CPU oracle (test infrastructure) into oracle/_build/libmsc_oracle.so.

The oracle is plain C built with IEEE semantics kept intact: no fast-math and no
floating-point contraction, so that every float operation is one correctly rounded
IEEE operation, exactly as the edit arithmetic (Eq. 2) is written.  Its per-cell loops
are OpenMP loops (-fopenmp); their results do not depend on the number of threads.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "msc_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmsc_oracle.so")


def build(force: bool = False) -> str:
    """Build the shared library if it is missing or older than its source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wno-unused-function", SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
