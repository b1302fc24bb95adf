"""The CUDA path's per-anchor gradient evaluator (eval_anchor and its compile-time cell
tables) and its pair decoder, compiled for the host, against the oracle on CPU: a check of
the device logic that needs no GPU (the GPU parity tests check the kernels themselves).
The same fields as the GPU gradient tests: random, all-equal, binary, signed-zero and
few-level values on 2D and 3D grids, boundary anchors included."""
import ctypes
import os
import shutil
import subprocess
import zlib

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "host_eval", "host_eval.cu")
OUT = os.path.join(HERE, "host_eval", "_build", "libhost_eval.so")
DEPS = [SRC] + [os.path.join(HERE, "..", "paper_2409_17346_gb300", "csrc", f) for f in ("msc_core.cuh", "msc_cells.cuh")]


@pytest.fixture(scope="module")
def lib():
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    if not os.path.exists(OUT) or any(os.path.getmtime(d) > os.path.getmtime(OUT) for d in DEPS):
        os.makedirs(os.path.dirname(OUT), exist_ok=True)
        tmp = OUT + ".tmp.%d" % os.getpid()
        subprocess.check_call([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode=arch=compute_103a,code=sm_103a",
                               "-O2", "-Xcompiler", "-fPIC", "-shared", "-o", tmp, SRC])
        os.replace(tmp, OUT)
    h = ctypes.CDLL(OUT)
    h.host_gradient_pairs.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
    return h


def _pairs(lib, a):
    a = np.ascontiguousarray(a, np.float32)
    ny, nx = a.shape[-2:]
    nz = a.shape[0] if a.ndim == 3 else 1
    n = ctypes.c_uint64(0)
    lib.host_gradient_pairs(a.ctypes.data, nx, ny, nz, None, 0, ctypes.byref(n))
    out = np.zeros((max(n.value, 1), 8), np.int64)
    lib.host_gradient_pairs(a.ctypes.data, nx, ny, nz, out.ctypes.data, n.value, ctypes.byref(n))
    out = out[: n.value]
    return out[np.lexsort(out.T[::-1])] if len(out) else out


def _field(shape, kind, rng):
    if kind == "normal":
        a = rng.standard_normal(shape)
    elif kind == "equal":
        a = np.zeros(shape)
    elif kind == "binary":
        a = rng.integers(0, 2, shape).astype(float)
    elif kind == "signed_zero":
        a = np.where(rng.random(shape) < 0.5, -0.0, 0.0) + (rng.random(shape) < 0.2)
    else:
        a = rng.integers(0, 4, shape).astype(float) * 0.25
    return a.astype(np.float32)


@pytest.mark.parametrize("shape", [(2, 2), (2, 9), (9, 2), (13, 11), (2, 2, 2), (2, 3, 5), (5, 4, 6), (7, 6, 5)])
@pytest.mark.parametrize("kind", ["normal", "equal", "binary", "signed_zero", "levels"])
def test_device_evaluator_matches_oracle_gradient(lib, shape, kind):
    rng = np.random.default_rng(zlib.crc32(repr((shape, kind)).encode()))
    a = _field(shape, kind, rng)
    assert np.array_equal(_pairs(lib, a), oracle.gradient_pairs(a))
