"""CPU oracle for the DMTz fix loop -- TEST INFRASTRUCTURE ONLY.

A plain, slow C restatement of the paper's method (see ``msc_oracle.c`` for the
passages each function follows), wrapped here with ctypes.  Only the test suite,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import this
package; the product path never does, and it shares no code with the CUDA path.

Fields are numpy float32 arrays of shape (ny, nx) for 2D or (nz, ny, nx) for 3D,
x fastest, so vertex id v = x + nx * (y + ny * z).
"""
import ctypes
import numpy as np

from . import build as _build

STATUS_OK = 0
ST_FLOOR = 0xF0
ST_EXACT = 0xF1

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
    return _lib


def set_threads(n):
    """Number of threads the oracle's parallel loops use (results do not depend on it)."""
    _load().orc_set_threads(int(n))


def threads():
    """Number of threads the oracle's parallel loops use."""
    return int(_load().orc_threads())


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(field):
    a = np.asarray(field)
    if a.ndim == 2:
        ny, nx = a.shape
        nz = 1
    elif a.ndim == 3:
        nz, ny, nx = a.shape
    else:
        raise ValueError("field must be 2D or 3D")
    return int(nx), int(ny), int(nz)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, rc))


def _sorted_rows(a):
    if len(a) == 0:
        return a
    order = np.lexsort(a.T[::-1])
    return a[order]


def gradient_pairs(field, brute=False):
    """All gradient pairs (L, U) as rows of 8 vertex ids, sorted (Sec. 4.2 / Sec. 3.1)."""
    lib = _load()
    f = _f32(field)
    nx, ny, nz = _dims(f)
    n = ctypes.c_int64(0)
    _check(lib.orc_gradient_pairs(_p(f), nx, ny, nz, int(brute), None, ctypes.c_int64(0), ctypes.byref(n)), "gradient")
    out = np.zeros((max(n.value, 1), 8), dtype=np.int64)
    _check(lib.orc_gradient_pairs(_p(f), nx, ny, nz, int(brute), _p(out), ctypes.c_int64(n.value), ctypes.byref(n)), "gradient")
    return _sorted_rows(out[: n.value])


def critical_cells(field):
    """Critical cells as (cells (n,4) vertex ids -1 padded, dims (n,)), sorted by cell."""
    lib = _load()
    f = _f32(field)
    nx, ny, nz = _dims(f)
    n = ctypes.c_int64(0)
    _check(lib.orc_critical_cells(_p(f), nx, ny, nz, None, None, ctypes.c_int64(0), ctypes.byref(n)), "critical")
    cells = np.zeros((max(n.value, 1), 4), dtype=np.int64)
    dims = np.zeros(max(n.value, 1), dtype=np.int32)
    _check(lib.orc_critical_cells(_p(f), nx, ny, nz, _p(cells), _p(dims), ctypes.c_int64(n.value), ctypes.byref(n)), "critical")
    cells, dims = cells[: n.value], dims[: n.value]
    if len(cells):
        order = np.lexsort(cells.T[::-1])
        cells, dims = cells[order], dims[order]
    return cells, dims


def cells(nx, ny, nz=1):
    """Every cell of the triangulated grid as rows of 4 vertex ids (-1 padded)."""
    lib = _load()
    n = ctypes.c_int64(0)
    _check(lib.orc_cells(nx, ny, nz, None, ctypes.c_int64(0), ctypes.byref(n)), "cells")
    out = np.zeros((max(n.value, 1), 4), dtype=np.int64)
    _check(lib.orc_cells(nx, ny, nz, _p(out), ctypes.c_int64(n.value), ctypes.byref(n)), "cells")
    return out[: n.value]


def separatrices(field, kind):
    """Separatrices of a field; kind 0 = descending, 1 = ascending.  Rows of 14:
    saddle (4 ids), start cell (4), path length, terminal (4), terminal dim."""
    lib = _load()
    f = _f32(field)
    nx, ny, nz = _dims(f)
    n = ctypes.c_int64(0)
    _check(lib.orc_separatrices(_p(f), nx, ny, nz, kind, None, ctypes.c_int64(0), ctypes.byref(n)), "separatrices")
    out = np.zeros((max(n.value, 1), 14), dtype=np.int64)
    _check(lib.orc_separatrices(_p(f), nx, ny, nz, kind, _p(out), ctypes.c_int64(n.value), ctypes.byref(n)), "separatrices")
    return out[: n.value]


def saddle_connectors(field):
    """The saddle-saddle walk of a 3D field's gradient from every 2-saddle.  Rows of 13:
    2-saddle (4 ids), kind (0 = 1-saddle edge reached, 1 = pair (edge, triangle) crossed,
    2 = dead-end edge paired down with a vertex), edge (4 ids), other cell (4 ids)."""
    lib = _load()
    f = _f32(field)
    nx, ny, nz = _dims(f)
    n = ctypes.c_int64(0)
    _check(lib.orc_saddle_connectors(_p(f), nx, ny, nz, None, ctypes.c_int64(0), ctypes.byref(n)), "saddle_connectors")
    out = np.zeros((max(n.value, 1), 13), dtype=np.int64)
    _check(lib.orc_saddle_connectors(_p(f), nx, ny, nz, _p(out), ctypes.c_int64(n.value), ctypes.byref(n)),
           "saddle_connectors")
    return out[: n.value]


def targets(f, g, state=None, pass_=0, tier=4, exact_fallback=1):
    """One targeting pass (0 = C-pass, 1 = S-pass) on (f, g, state).  Returns
    (cases: rows (target vertex, case cell 4 ids), markX: uint8 per vertex)."""
    lib = _load()
    f = _f32(f)
    g = _f32(g)
    nx, ny, nz = _dims(f)
    n_v = f.size
    st = np.zeros(n_v, dtype=np.uint8) if state is None else np.ascontiguousarray(state, dtype=np.uint8).reshape(-1)
    cap = 26 * n_v + 16
    out = np.zeros((cap, 5), dtype=np.int64)
    markX = np.zeros(n_v, dtype=np.uint8)
    n = ctypes.c_int64(0)
    _check(lib.orc_targets(_p(f), _p(g), _p(st), nx, ny, nz, pass_, tier, exact_fallback,
                           _p(out), ctypes.c_int64(cap), ctypes.byref(n), _p(markX)), "targets")
    return out[: min(n.value, cap)], markX


def fix(f, fhat, xi, tier=4, q_max=6, max_iters=100000, exact_fallback=1, trace_cap=1 << 20, edit_mode=0):
    """The whole fix loop.  edit_mode 0: quantised edits (Eq. 2); 1: floating edits (no cap
    on the number of steps, Sec. 4.7).  Returns a dict with g, state, n_c, n_s,
    n_exact_iters, trace (rows: kind, |T|, |X|, sum T, sum X, #cases) and status."""
    lib = _load()
    f = _f32(f)
    fhat = _f32(fhat)
    if f.shape != fhat.shape:
        raise ValueError("shape mismatch")
    nx, ny, nz = _dims(f)
    g = np.zeros_like(f)
    state = np.zeros(f.shape, dtype=np.uint8)
    counts = np.zeros(3, dtype=np.int32)
    trace = np.zeros((trace_cap, 6), dtype=np.int64)
    ntr = ctypes.c_int64(0)
    rc = lib.orc_fix(_p(f), _p(fhat), nx, ny, nz, ctypes.c_float(xi), tier, q_max, max_iters,
                     exact_fallback, edit_mode, _p(g), _p(state), _p(counts), _p(trace),
                     ctypes.c_int64(trace_cap), ctypes.byref(ntr))
    return dict(status=rc, g=g, state=state, n_c=int(counts[0]), n_s=int(counts[1]),
                n_exact_iters=int(counts[2]), trace=trace[: min(ntr.value, trace_cap)])


REPORT_KEYS = ("fp0", "fp1", "fp2", "fp3", "fn0", "fn1", "fn2", "fn3",
               "sep_desc", "sep_asc", "sep_saddle", "term_desc", "term_asc")


def verify(f, g):
    """MSC comparison of g against f; returns dict of the 13 report counts + max_abs_err."""
    lib = _load()
    f = _f32(f)
    g = _f32(g)
    nx, ny, nz = _dims(f)
    rep = np.zeros(13, dtype=np.int64)
    err = ctypes.c_double(0.0)
    _check(lib.orc_verify(_p(f), _p(g), nx, ny, nz, _p(rep), ctypes.byref(err)), "verify")
    out = {k: int(v) for k, v in zip(REPORT_KEYS, rep)}
    out["max_abs_err"] = err.value
    return out


def edit_values(f, fhat, xi, q_max=6, n_steps=None):
    """Closed-form pieces of Eq. 2: (lb, ub, clamped base, values after q = 0 .. n_steps - 1
    steps of xi / 2^q_max); n_steps defaults to q_max + 1."""
    lib = _load()
    f = _f32(f).reshape(-1)
    fhat = _f32(fhat).reshape(-1)
    n = f.size
    nq = q_max + 1 if n_steps is None else int(n_steps)
    lb = np.zeros(n, np.float32)
    ub = np.zeros(n, np.float32)
    fc = np.zeros(n, np.float32)
    qv = np.zeros((n, nq), np.float32)
    _check(lib.orc_edit_values(_p(f), _p(fhat), ctypes.c_int64(n), ctypes.c_float(xi), q_max, nq,
                               _p(lb), _p(ub), _p(fc), _p(qv)), "edit_values")
    return lb, ub, fc, qv


def apply_edits(fhat, xi, q_max, q_map, lossless_idx, lossless_val):
    """Decompression side: rebuild g from fhat and the stored edits."""
    lib = _load()
    fh = _f32(fhat)
    qm = np.ascontiguousarray(q_map, dtype=np.uint8).reshape(-1)
    li = np.ascontiguousarray(lossless_idx, dtype=np.int64).reshape(-1)
    lv = np.ascontiguousarray(lossless_val, dtype=np.float32).reshape(-1)
    g = np.zeros_like(fh)
    _check(lib.orc_apply_edits(_p(fh), ctypes.c_int64(fh.size), ctypes.c_float(xi), q_max, _p(qm),
                               _p(li), _p(lv), ctypes.c_int64(li.size), _p(g)), "apply_edits")
    return g


def edits_from_state(f, fhat, xi, state, g, edit_mode=0):
    """The stored form of the edits (Sec. 4.7): q per quantised vertex; 0xFF and the exact
    final value for floor, exact, or re-clamped vertices.  Floating edits (edit_mode 1) store
    every edited vertex that way."""
    f = _f32(f).reshape(-1)
    fhat = _f32(fhat).reshape(-1)
    st = np.asarray(state, dtype=np.uint8).reshape(-1)
    gg = _f32(g).reshape(-1)
    _, _, fc, _ = edit_values(f, fhat, xi, 1)
    clamped = fc.view(np.uint32) != fhat.view(np.uint32)
    lossless = (st > (0 if edit_mode else 7)) | clamped
    q_map = np.where(lossless, 0xFF, st).astype(np.uint8)
    idx = np.nonzero(lossless)[0].astype(np.int64)
    return q_map, idx, gg[idx].copy()


def packed_bytes(n, n_lossless, q_max):
    """Size of the packed edit record (Sec. 4.7)."""
    lib = _load()
    lib.orc_packed_bytes.restype = ctypes.c_int64
    return int(lib.orc_packed_bytes(ctypes.c_int64(n), ctypes.c_int64(n_lossless), q_max))


def pack_edits(q_map, q_max, lossless_val):
    """The edit record as bytes: header, q-map at a fixed number of bits per vertex, lossless
    values in increasing vertex order."""
    lib = _load()
    qm = np.ascontiguousarray(q_map, dtype=np.uint8).reshape(-1)
    lv = np.ascontiguousarray(lossless_val, dtype=np.float32).reshape(-1)
    size = packed_bytes(qm.size, lv.size, q_max)
    out = np.zeros(size, np.uint8)
    n_out = ctypes.c_int64(0)
    _check(lib.orc_pack_edits(_p(qm), ctypes.c_int64(qm.size), q_max, _p(lv), ctypes.c_int64(lv.size), _p(out),
                              ctypes.c_int64(size), ctypes.byref(n_out)), "pack_edits")
    return out


def unpack_edits(buf):
    """Inverse of pack_edits: (q_map, lossless_idx, lossless_val, q_max)."""
    lib = _load()
    b = np.ascontiguousarray(buf, dtype=np.uint8).reshape(-1)
    n, nl, qmax = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int(0)
    _check(lib.orc_packed_header(_p(b), ctypes.c_int64(b.size), ctypes.byref(n), ctypes.byref(nl),
                                 ctypes.byref(qmax)), "unpack_edits")
    qm = np.zeros(n.value, np.uint8)
    li = np.zeros(nl.value, np.int64)
    lv = np.zeros(nl.value, np.float32)
    _check(lib.orc_unpack_edits(_p(b), ctypes.c_int64(b.size), _p(qm), _p(li), _p(lv)), "unpack_edits")
    return qm, li, lv, qmax.value
