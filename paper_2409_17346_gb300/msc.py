"""Thin Python binding of libmsc (include/msc.h): argument marshalling only.

Every computation runs in the CUDA library.  Fields may be numpy arrays (host memory) or
torch CUDA tensors (device memory, passed by pointer); both must be float32, C-contiguous,
shape (ny, nx) or (nz, ny, nx).  The binding raises ``MscError`` on any status other than
MSC_OK, and ``RuntimeError`` if the library has not been built.
"""
import ctypes
import os

import numpy as np

from . import build as _build

MSC_OK = 0
STATUS_NAMES = {0: "MSC_OK", 1: "MSC_ERR_INVALID_ARG", 2: "MSC_ERR_OOM", 3: "MSC_ERR_CUDA",
                4: "MSC_ERR_NOT_CONVERGED", 5: "MSC_ERR_DEVICE_TIMEOUT", 6: "MSC_ERR_STALLED",
                7: "MSC_ERR_NO_DEVICE", 8: "MSC_ERR_CANCELLED", 9: "MSC_ERR_UNAVAILABLE"}
QMAP_LOSSLESS = 0xFF


class MscError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("tier", ctypes.c_int), ("q_max", ctypes.c_int), ("max_iters", ctypes.c_int),
                ("exact_fallback", ctypes.c_int), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
                ("tile_z", ctypes.c_int), ("stream", ctypes.c_void_p), ("record_trace", ctypes.c_int),
                ("profile", ctypes.c_int), ("small_round", ctypes.c_int), ("edit_mode", ctypes.c_int),
                ("cluster_round", ctypes.c_int)]


KERNEL_CLASSES = ("dense", "cpass", "edit", "refresh", "rebuild", "sep_init", "sep_update", "sep_targets", "other",
                  "sep_seed", "rounds")
PROFILE_ALL = (1 << len(KERNEL_CLASSES)) - 1


def profile_mask(profile):
    """options.profile from True/False (all/no classes), a class name, an iterable of class
    names, or an integer bitmask."""
    if profile is True:
        return PROFILE_ALL
    if not profile:
        return 0
    if isinstance(profile, str):
        return 1 << KERNEL_CLASSES.index(profile)
    if isinstance(profile, int):
        return profile & PROFILE_ALL
    return sum(1 << KERNEL_CLASSES.index(k) for k in set(profile))


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64 * 12), ("ms", ctypes.c_double * 12),
                ("timed_launches", ctypes.c_uint64 * 12), ("items", ctypes.c_uint64 * 12),
                ("round_work", ctypes.c_uint64 * 3), ("round_phase_ms", ctypes.c_double * 4),
                ("cluster_launches", ctypes.c_uint64), ("cluster_rounds", ctypes.c_uint64)]


class IterRecord(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("t_us", ctypes.c_int32), ("n_targets", ctypes.c_int64),
                ("n_exact", ctypes.c_int64), ("sum_targets", ctypes.c_int64), ("sum_exact", ctypes.c_int64)]


class Edits(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_uint64), ("n_iters_c", ctypes.c_uint32), ("n_iters_s", ctypes.c_uint32),
                ("n_fallback_iters", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("n_quant", ctypes.c_uint64), ("n_lossless", ctypes.c_uint64),
                ("q_map", ctypes.POINTER(ctypes.c_uint8)), ("lossless_idx", ctypes.POINTER(ctypes.c_uint64)),
                ("lossless_val", ctypes.POINTER(ctypes.c_float)), ("n_trace", ctypes.c_uint32),
                ("trace", ctypes.POINTER(IterRecord)), ("loop_ms", ctypes.c_double)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_jobs", ctypes.c_int), ("max_skips", ctypes.c_int), ("mem_budget", ctypes.c_uint64),
                ("options", Options)]


class JobInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("slot", ctypes.c_int32), ("bytes", ctypes.c_uint64),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_end", ctypes.c_double),
                ("loop_ms", ctypes.c_float), ("reserved", ctypes.c_uint32)]


class Report(ctypes.Structure):
    _fields_ = [("fp", ctypes.c_uint64 * 4), ("fn", ctypes.c_uint64 * 4), ("sep_mismatch", ctypes.c_uint64 * 3),
                ("term_mismatch", ctypes.c_uint64 * 2), ("max_abs_err", ctypes.c_double), ("pass_", ctypes.c_int),
                ("pass_tier", ctypes.c_int * 4), ("reserved", ctypes.c_int)]


_lib = None


def library_path():
    return _build.LIB


def load():
    """Load libmsc.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libmsc is not built (%s missing): run __graft_entry__.build()" % _build.LIB)
    lib = ctypes.CDLL(_build.LIB)
    vp, i, f, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_uint64
    lib.msc_version.restype = ctypes.c_char_p
    lib.msc_status_string.restype = ctypes.c_char_p
    lib.msc_status_string.argtypes = [i]
    lib.msc_last_error.restype = ctypes.c_char_p
    lib.msc_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.msc_prepare_original.argtypes = [vp, i, i, i, ctypes.POINTER(Options), ctypes.POINTER(vp)]
    lib.msc_fix.argtypes = [vp, vp, f, ctypes.POINTER(Options), ctypes.POINTER(Edits), vp]
    lib.msc_apply_edits.argtypes = [vp, i, i, i, f, i, ctypes.POINTER(Edits), vp]
    lib.msc_verify.argtypes = [vp, vp, f, ctypes.POINTER(Report)]
    lib.msc_free_edits.argtypes = [ctypes.POINTER(Edits)]
    lib.msc_free_edits.restype = None
    lib.msc_destroy.argtypes = [vp]
    lib.msc_destroy.restype = None
    lib.msc_fix_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(f), i,
                                  ctypes.POINTER(Options), ctypes.POINTER(Edits), ctypes.POINTER(vp)]
    lib.msc_gradient_pairs.argtypes = [vp, i, i, i, vp, u64, ctypes.POINTER(u64)]
    lib.msc_critical_cells.argtypes = [vp, i, i, i, vp, vp, u64, ctypes.POINTER(u64)]
    lib.msc_critical_cells_static.argtypes = [vp, i, i, i, vp, vp, u64, ctypes.POINTER(u64), vp]
    lib.msc_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    lib.msc_server_submit.argtypes = [vp, vp, vp, i, i, i, f, vp, ctypes.POINTER(u64)]
    lib.msc_server_wait.argtypes = [vp, u64, ctypes.POINTER(Edits), ctypes.POINTER(JobInfo)]
    lib.msc_server_destroy.argtypes = [vp]
    lib.msc_server_destroy.restype = None
    lib.msc_packed_bytes.argtypes = [u64, u64, i]
    lib.msc_packed_bytes.restype = u64
    lib.msc_pack_edits.argtypes = [ctypes.POINTER(Edits), i, vp, u64, ctypes.POINTER(u64)]
    lib.msc_unpack_edits.argtypes = [vp, u64, ctypes.POINTER(Edits), ctypes.POINTER(i)]
    lib.msc_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.msc_reset_stats.argtypes = [vp]
    lib.msc_device_bytes.argtypes = [i, i, i]
    lib.msc_device_bytes.restype = u64
    lib.msc_selftest_barrier.argtypes = [i, vp]
    lib.msc_release_cached_memory.argtypes = []
    lib.msc_pool_used_bytes.argtypes = [ctypes.POINTER(u64)]
    lib.msc_set_walk_limits.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
    lib.msc_set_walk_limits.restype = ctypes.c_int
    lib.msc_inject_alloc_failures.argtypes = [u64, u64]
    lib.msc_inject_alloc_failures.restype = u64
    lib.msc_server_cancel.argtypes = [vp, u64]
    lib.msc_tile_report.argtypes = [i, i, i, vp, vp, vp, i, ctypes.POINTER(i)]
    lib.msc_kv_bytes.argtypes = [u64]
    lib.msc_kv_bytes.restype = u64
    lib.msc_pack_edits_kv.argtypes = [ctypes.POINTER(Edits), vp, u64, ctypes.POINTER(u64)]
    lib.msc_unpack_edits_kv.argtypes = [vp, u64, ctypes.POINTER(Edits)]
    lib.msc_coded_bound.argtypes = [u64]
    lib.msc_coded_bound.restype = u64
    lib.msc_code_record.argtypes = [vp, u64, i, vp, u64, ctypes.POINTER(u64)]
    lib.msc_decoded_size.argtypes = [vp, u64, ctypes.POINTER(u64)]
    lib.msc_decode_record.argtypes = [vp, u64, vp, u64, ctypes.POINTER(u64)]
    for name in ("msc_prepare_original", "msc_fix", "msc_apply_edits", "msc_verify", "msc_fix_batch",
                 "msc_gradient_pairs", "msc_critical_cells", "msc_critical_cells_static", "msc_get_stats",
                 "msc_reset_stats", "msc_server_create", "msc_server_submit", "msc_server_wait", "msc_pack_edits",
                 "msc_unpack_edits", "msc_pool_used_bytes", "msc_release_cached_memory", "msc_selftest_barrier",
                 "msc_server_cancel", "msc_pack_edits_kv", "msc_unpack_edits_kv", "msc_code_record",
                 "msc_decoded_size", "msc_decode_record", "msc_tile_report"):
        getattr(lib, name).restype = i
    _lib = lib
    return lib


def _check(status):
    if status != MSC_OK:
        raise MscError(status, load().msc_last_error().decode())


def dims_of(shape):
    if len(shape) == 2:
        return int(shape[1]), int(shape[0]), 1
    if len(shape) == 3:
        return int(shape[2]), int(shape[1]), int(shape[0])
    raise ValueError("field must be 2D (ny, nx) or 3D (nz, ny, nx)")


def _ptr(a):
    """(pointer, keepalive) of a float32 numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.float32)
        return a.ctypes.data_as(ctypes.c_void_p), a
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise ValueError("tensors must be contiguous float32")
        return ctypes.c_void_p(a.data_ptr()), a
    raise TypeError("expected a numpy array or a torch tensor")


EDITS_QUANTIZED, EDITS_FLOAT = 0, 1


def options(tier=4, q_max=6, max_iters=100000, exact_fallback=1, stream=None, record_trace=False,
            tile=(0, 0, 0), profile=False, small_round=0, edit_mode=EDITS_QUANTIZED, cluster_round=0):
    o = Options()
    load().msc_default_options(ctypes.byref(o))
    o.tier, o.q_max, o.max_iters, o.exact_fallback = tier, q_max, max_iters, exact_fallback
    o.tile_x, o.tile_y, o.tile_z = tile
    o.stream = ctypes.c_void_p(stream) if stream else None
    o.record_trace = int(bool(record_trace))
    o.profile = profile_mask(profile)
    o.small_round = small_round
    o.edit_mode = int(edit_mode)
    o.cluster_round = int(cluster_round)
    return o


class _EditsOwner:
    """Owns one msc_edits record; msc_free_edits runs when the last array viewing it goes."""

    def __init__(self, e):
        self.e = e

    def __del__(self):
        try:
            load().msc_free_edits(ctypes.byref(self.e))
        except Exception:
            pass


def _view(ptr, count, ctype, dtype, owner):
    """A numpy array over count elements at ptr; it keeps owner alive."""
    buf = (ctype * count).from_address(ctypes.cast(ptr, ctypes.c_void_p).value)
    buf._owner = owner
    return np.frombuffer(buf, dtype=dtype)


_TRACE_DTYPE = np.dtype([("kind", np.int32), ("t_us", np.int32), ("n_targets", np.int64), ("n_exact", np.int64),
                         ("sum_targets", np.int64), ("sum_exact", np.int64)])


def _edits_to_py(e, shape, owner=None):
    """The record as a dict of numpy arrays: copies, or (owner given) views of the library's
    buffers that free the record once the last of them is gone."""
    n = int(e.n_vertices)
    out = dict(n_iters_c=int(e.n_iters_c), n_iters_s=int(e.n_iters_s), n_fallback_iters=int(e.n_fallback_iters),
               n_quant=int(e.n_quant), n_lossless=int(e.n_lossless), loop_ms=float(e.loop_ms))
    nl = int(e.n_lossless)
    if owner is None:
        out["q_map"] = np.ctypeslib.as_array(e.q_map, shape=(n,)).copy().reshape(shape) if n else np.zeros(shape, np.uint8)
        out["lossless_idx"] = np.ctypeslib.as_array(e.lossless_idx, shape=(nl,)).copy() if nl else np.zeros(0, np.uint64)
        out["lossless_val"] = np.ctypeslib.as_array(e.lossless_val, shape=(nl,)).copy() if nl else np.zeros(0, np.float32)
    else:
        out["q_map"] = _view(e.q_map, n, ctypes.c_uint8, np.uint8, owner).reshape(shape) if n else np.zeros(shape, np.uint8)
        out["lossless_idx"] = _view(e.lossless_idx, nl, ctypes.c_uint64, np.uint64, owner) if nl else np.zeros(0, np.uint64)
        out["lossless_val"] = _view(e.lossless_val, nl, ctypes.c_float, np.float32, owner) if nl else np.zeros(0, np.float32)
    nt = int(e.n_trace)
    if nt:
        raw = np.frombuffer((ctypes.c_uint8 * (nt * _TRACE_DTYPE.itemsize)).from_address(
            ctypes.cast(e.trace, ctypes.c_void_p).value), dtype=_TRACE_DTYPE).copy()
        out["trace"] = np.stack([raw["kind"].astype(np.int64), raw["n_targets"], raw["n_exact"], raw["sum_targets"],
                                 raw["sum_exact"]], axis=1)
        out["trace_t_us"] = raw["t_us"].astype(np.int64)
    else:
        out["trace"] = np.zeros((0, 5), np.int64)
        out["trace_t_us"] = np.zeros(0, np.int64)
    return out


class Handle:
    """Device-resident MSC of one original field f (msc_prepare_original)."""

    def __init__(self, f, opts=None, **kw):
        lib = load()
        if opts is None and kw:
            opts = options(**kw)
        self.shape = tuple(f.shape)
        self.nx, self.ny, self.nz = dims_of(self.shape)
        p, keep = _ptr(f)
        h = ctypes.c_void_p()
        _check(lib.msc_prepare_original(p, self.nx, self.ny, self.nz,
                                        ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().msc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def fix(self, f_hat, xi, g_out=None, **kw):
        """Run the fix loop; returns (g, edits dict).  g_out: optional torch CUDA tensor or
        numpy array receiving the corrected field."""
        lib = load()
        opts = options(**kw)
        p, keep = _ptr(f_hat)
        if g_out is None:
            g_out = np.zeros(self.shape, np.float32)
        gp, gkeep = _ptr(g_out)
        e = Edits()
        try:
            _check(lib.msc_fix(self._h, p, ctypes.c_float(xi), ctypes.byref(opts), ctypes.byref(e), gp))
        except BaseException:
            lib.msc_free_edits(ctypes.byref(e))
            raise
        return g_out, _edits_to_py(e, self.shape, _EditsOwner(e))

    def stats(self):
        """Launch counts and profiled CUDA-event milliseconds by kernel class."""
        st = Stats()
        _check(load().msc_get_stats(self._h, ctypes.byref(st)))
        out = {k: dict(launches=int(st.launches[i]), ms=float(st.ms[i]), timed=int(st.timed_launches[i]),
                       items=int(st.items[i]))
               for i, k in enumerate(KERNEL_CLASSES)}
        out["rounds"]["work"] = dict(edit=int(st.round_work[0]), refresh=int(st.round_work[1]),
                                     cpass=int(st.round_work[2]))
        out["rounds"]["phase_ms"] = dict(zip(("cpass", "edit", "mark", "refresh"),
                                             (float(v) for v in st.round_phase_ms)))
        out["rounds"]["cluster_launches"] = int(st.cluster_launches)
        out["rounds"]["cluster_rounds"] = int(st.cluster_rounds)
        return out

    def reset_stats(self):
        _check(load().msc_reset_stats(self._h))

    def verify(self, g, xi):
        lib = load()
        p, keep = _ptr(g)
        r = Report()
        _check(lib.msc_verify(self._h, p, ctypes.c_float(xi), ctypes.byref(r)))
        return dict(fp=list(r.fp), fn=list(r.fn), sep_mismatch=list(r.sep_mismatch),
                    term_mismatch=list(r.term_mismatch), max_abs_err=r.max_abs_err, passed=bool(r.pass_),
                    passed_tier=[bool(x) for x in r.pass_tier])


def apply_edits(f_hat, xi, q_max, edits, g_out=None):
    """Decompression side: rebuild g from f_hat and the edits returned by Handle.fix."""
    lib = load()
    shape = tuple(f_hat.shape)
    nx, ny, nz = dims_of(shape)
    e = Edits()
    qm = np.ascontiguousarray(edits["q_map"], dtype=np.uint8).reshape(-1)
    li = np.ascontiguousarray(edits["lossless_idx"], dtype=np.uint64)
    lv = np.ascontiguousarray(edits["lossless_val"], dtype=np.float32)
    e.n_vertices = qm.size
    e.n_lossless = li.size
    e.q_map = qm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    e.lossless_idx = li.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    e.lossless_val = lv.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    p, keep = _ptr(f_hat)
    if g_out is None:
        g_out = np.zeros(shape, np.float32)
    gp, gkeep = _ptr(g_out)
    _check(lib.msc_apply_edits(p, nx, ny, nz, ctypes.c_float(xi), q_max, ctypes.byref(e), gp))
    return g_out


def _edits_struct(edits):
    """An Edits view of an edits dict (the arrays stay owned by the dict)."""
    qm = np.ascontiguousarray(edits["q_map"], dtype=np.uint8).reshape(-1)
    li = np.ascontiguousarray(edits["lossless_idx"], dtype=np.uint64)
    lv = np.ascontiguousarray(edits["lossless_val"], dtype=np.float32)
    e = Edits()
    e.n_vertices = qm.size
    e.n_lossless = li.size
    e.n_quant = int(np.count_nonzero((qm != 0) & (qm != QMAP_LOSSLESS)))
    e.q_map = qm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    e.lossless_idx = li.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    e.lossless_val = lv.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    return e, (qm, li, lv)


def packed_bytes(n_vertices, n_lossless, q_max):
    return int(load().msc_packed_bytes(n_vertices, n_lossless, q_max))


def pack_edits(edits, q_max):
    """msc_pack_edits: the edit record as a uint8 array (Sec. 4.7 fixed-bit q-map)."""
    lib = load()
    e, keep = _edits_struct(edits)
    n = ctypes.c_uint64(0)
    _check(lib.msc_pack_edits(ctypes.byref(e), q_max, None, 0, ctypes.byref(n)))
    out = np.zeros(n.value, np.uint8)
    _check(lib.msc_pack_edits(ctypes.byref(e), q_max, out.ctypes.data_as(ctypes.c_void_p), out.size, ctypes.byref(n)))
    return out


def unpack_edits(buf, shape):
    """msc_unpack_edits: (edits dict, q_max) from a packed record."""
    lib = load()
    b = np.ascontiguousarray(buf, dtype=np.uint8).reshape(-1)
    e = Edits()
    q = ctypes.c_int(0)
    try:
        _check(lib.msc_unpack_edits(b.ctypes.data_as(ctypes.c_void_p), b.size, ctypes.byref(e), ctypes.byref(q)))
        out = _edits_to_py(e, tuple(shape))
    finally:
        lib.msc_free_edits(ctypes.byref(e))
    return out, q.value


def pack_edits_kv(edits):
    """Floating edits (edit_mode 1) as a key-value record (numpy uint8 array)."""
    lib = load()
    e, _keep = _edits_struct(edits)
    n = ctypes.c_uint64(0)
    _check(lib.msc_pack_edits_kv(ctypes.byref(e), None, 0, ctypes.byref(n)))
    out = np.zeros(n.value, np.uint8)
    _check(lib.msc_pack_edits_kv(ctypes.byref(e), out.ctypes.data_as(ctypes.c_void_p), n.value, ctypes.byref(n)))
    return out


def unpack_edits_kv(buf, shape):
    """Edit record (dict as Handle.fix returns) from a key-value record."""
    lib = load()
    b = np.ascontiguousarray(buf, np.uint8)
    e = Edits()
    _check(lib.msc_unpack_edits_kv(b.ctypes.data_as(ctypes.c_void_p), b.size, ctypes.byref(e)))
    return _edits_to_py(e, shape, _EditsOwner(e))


def code_record(rec, level=3):
    """Lossless coding of a record (zstd frame, Sec. 4.7 / 5.5): numpy uint8 array."""
    lib = load()
    r = np.ascontiguousarray(rec, np.uint8)
    cap = int(lib.msc_coded_bound(r.size))
    if cap == 0:
        _check(lib.msc_code_record(None, 0, level, None, 0, ctypes.byref(ctypes.c_uint64(0))))
    out = np.zeros(cap, np.uint8)
    n = ctypes.c_uint64(0)
    _check(lib.msc_code_record(r.ctypes.data_as(ctypes.c_void_p), r.size, int(level),
                               out.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(n)))
    return out[: n.value].copy()


def decode_record(coded):
    """Inverse of code_record."""
    lib = load()
    c = np.ascontiguousarray(coded, np.uint8)
    n = ctypes.c_uint64(0)
    _check(lib.msc_decoded_size(c.ctypes.data_as(ctypes.c_void_p), c.size, ctypes.byref(n)))
    out = np.zeros(max(n.value, 1), np.uint8)
    _check(lib.msc_decode_record(c.ctypes.data_as(ctypes.c_void_p), c.size, out.ctypes.data_as(ctypes.c_void_p),
                                 out.size, ctypes.byref(n)))
    return out[: n.value]


def fix_batch(handles, f_hats, xis, g_outs=None, **kw):
    """msc_fix_batch over several jobs; returns (list of g, list of edit dicts)."""
    lib = load()
    n = len(handles)
    opts = options(**kw)
    if g_outs is None:
        g_outs = [np.zeros(h.shape, np.float32) for h in handles]
    hp = (ctypes.c_void_p * n)(*[h._h.value for h in handles])
    fps, keeps = [], []
    for a in f_hats:
        p, k = _ptr(a)
        fps.append(p.value)
        keeps.append(k)
    gps = []
    for a in g_outs:
        p, k = _ptr(a)
        gps.append(p.value)
        keeps.append(k)
    fp = (ctypes.c_void_p * n)(*fps)
    gp = (ctypes.c_void_p * n)(*gps)
    xa = (ctypes.c_float * n)(*[float(x) for x in xis])
    es = (Edits * n)()
    try:
        _check(lib.msc_fix_batch(hp, fp, xa, n, ctypes.byref(opts), es, gp))
    except BaseException:
        for i in range(n):
            lib.msc_free_edits(ctypes.byref(es[i]))
        raise
    outs = []
    for i in range(n):
        e = Edits()
        ctypes.memmove(ctypes.byref(e), ctypes.byref(es[i]), ctypes.sizeof(Edits))
        outs.append(_edits_to_py(e, handles[i].shape, _EditsOwner(e)))
    return g_outs, outs


class Server:
    """msc_server: continuous batching of fix jobs on the current device.

    submit() queues a job and returns its ticket at once; wait(ticket) blocks until that job
    is done and returns (g, edits dict, info dict).  The arrays passed to submit are kept
    alive here until their job has been waited for."""

    def __init__(self, max_jobs=8, mem_budget=0, max_skips=0, **opts):
        lib = load()
        cfg = ServerConfig()
        cfg.max_jobs, cfg.max_skips, cfg.mem_budget = int(max_jobs), int(max_skips), int(mem_budget)
        cfg.options = options(**opts)
        self._s = ctypes.c_void_p()
        _check(lib.msc_server_create(ctypes.byref(cfg), ctypes.byref(self._s)))
        self._jobs = {}

    def submit(self, f, f_hat, xi, g_out=None):
        lib = load()
        if g_out is None:
            g_out = np.zeros(np.shape(f), np.float32)
        fp, fk = _ptr(f)
        hp, hk = _ptr(f_hat)
        gp, gk = _ptr(g_out)
        nx, ny, nz = dims_of(np.shape(f))
        t = ctypes.c_uint64(0)
        _check(lib.msc_server_submit(self._s, fp, hp, nx, ny, nz, ctypes.c_float(xi), gp, ctypes.byref(t)))
        self._jobs[t.value] = (g_out, (fk, hk, gk), tuple(np.shape(f)))
        return t.value

    def cancel(self, ticket):
        """Cancel a queued or running job; its wait() then raises MscError (MSC_ERR_CANCELLED)."""
        _check(load().msc_server_cancel(self._s, ctypes.c_uint64(ticket)))

    def wait(self, ticket):
        lib = load()
        g_out, _keep, shape = self._jobs[ticket]
        e = Edits()
        info = JobInfo()
        try:
            st = lib.msc_server_wait(self._s, ticket, ctypes.byref(e), ctypes.byref(info))
            del self._jobs[ticket]
            _check(st)
            out = _edits_to_py(e, shape)
        finally:
            lib.msc_free_edits(ctypes.byref(e))
        inf = dict(status=int(info.status), slot=int(info.slot), bytes=int(info.bytes), t_submit=info.t_submit,
                   t_start=info.t_start, t_end=info.t_end, loop_ms=float(info.loop_ms))
        return g_out, out, inf

    def close(self):
        if self._s:
            load().msc_server_destroy(self._s)
            self._s = ctypes.c_void_p()
            self._jobs.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _sorted_rows(a):
    return a[np.lexsort(a.T[::-1])] if len(a) else a


def gradient_pairs(field):
    """All gradient pairs (L, U) of a host field as sorted rows of 8 vertex ids."""
    lib = load()
    f = np.ascontiguousarray(field, dtype=np.float32)
    nx, ny, nz = dims_of(f.shape)
    n = ctypes.c_uint64(0)
    _check(lib.msc_gradient_pairs(f.ctypes.data_as(ctypes.c_void_p), nx, ny, nz, None, 0, ctypes.byref(n)))
    rows = np.zeros((max(n.value, 1), 8), np.int64)
    _check(lib.msc_gradient_pairs(f.ctypes.data_as(ctypes.c_void_p), nx, ny, nz, rows.ctypes.data_as(ctypes.c_void_p),
                                  n.value, ctypes.byref(n)))
    return _sorted_rows(rows[: n.value])


def critical_cells(field):
    """Critical cells of a host field: (rows (n,4) sorted, dims (n,))."""
    lib = load()
    f = np.ascontiguousarray(field, dtype=np.float32)
    nx, ny, nz = dims_of(f.shape)
    n = ctypes.c_uint64(0)
    _check(lib.msc_critical_cells(f.ctypes.data_as(ctypes.c_void_p), nx, ny, nz, None, None, 0, ctypes.byref(n)))
    rows = np.zeros((max(n.value, 1), 4), np.int64)
    dims = np.zeros(max(n.value, 1), np.int32)
    _check(lib.msc_critical_cells(f.ctypes.data_as(ctypes.c_void_p), nx, ny, nz, rows.ctypes.data_as(ctypes.c_void_p),
                                  dims.ctypes.data_as(ctypes.c_void_p), n.value, ctypes.byref(n)))
    rows, dims = rows[: n.value], dims[: n.value]
    if len(rows):
        o = np.lexsort(rows.T[::-1])
        rows, dims = rows[o], dims[o]
    return rows, dims


STATIC_MAX_VERTICES = 1 << 20


def critical_cells_static(field_ptr, shape, rows_ptr, dims_ptr, cap, stream=None):
    """msc_critical_cells_static on caller-owned device buffers (integer addresses):
    field (float32, shape), rows (cap x 4 int64), dims (cap int32).  Returns the number
    of critical cells; at most cap rows are written, unordered."""
    nx, ny, nz = dims_of(shape)
    n = ctypes.c_uint64(0)
    _check(load().msc_critical_cells_static(field_ptr, nx, ny, nz, rows_ptr, dims_ptr, cap, ctypes.byref(n), stream))
    return n.value


def tile_report(shape):
    """The tile autotuner's record for a 3D grid on the current device: dict with the
    instantiated shapes, their times on the tuning pass (ms) and the shape kept (None if the
    grid was not tuned yet)."""
    lib = load()
    nx, ny, nz = dims_of(shape)
    n = ctypes.c_int(0)
    _check(lib.msc_tile_report(nx, ny, nz, None, None, None, 0, ctypes.byref(n)))
    chosen = np.zeros(3, np.int32)
    shapes = np.zeros((n.value, 3), np.int32)
    ms = np.zeros(n.value, np.float32)
    _check(lib.msc_tile_report(nx, ny, nz, chosen.ctypes.data_as(ctypes.c_void_p), shapes.ctypes.data_as(ctypes.c_void_p),
                               ms.ctypes.data_as(ctypes.c_void_p), n.value, ctypes.byref(n)))
    return {"shapes": [tuple(int(v) for v in r) for r in shapes], "ms": [float(v) for v in ms],
            "chosen": tuple(int(v) for v in chosen) if chosen[0] else None}


def device_bytes(shape):
    return int(load().msc_device_bytes(*dims_of(shape)))


def selftest_barrier(timeout_ms=100):
    """Status of msc_selftest_barrier (MSC_ERR_DEVICE_TIMEOUT = 5 is the expected outcome)."""
    return int(load().msc_selftest_barrier(int(timeout_ms), None))


def release_cached_memory():
    """Return the device memory the library's pool keeps for reuse to the driver."""
    _check(load().msc_release_cached_memory())


def inject_alloc_failures(after, count):
    """Test hook: after `after` more device allocations succeed, the next `count` fail as if
    the device were out of memory (count 0 turns it off).  Returns failures injected so far."""
    return int(load().msc_inject_alloc_failures(int(after), int(count)))


def set_walk_limits(warp_stack=0, local_steps=0):
    """Test hook: lower the saddle-saddle walk's per-warp stack (1..384 entries) and the steps
    one thread walks before it spills, so that small fields take the spill paths (0 restores
    a default).  Results do not depend on them."""
    _check(load().msc_set_walk_limits(int(warp_stack), int(local_steps)))


def pool_used_bytes():
    """Bytes of the library's device memory pool (current device) held by live buffers."""
    n = ctypes.c_uint64(0)
    _check(load().msc_pool_used_bytes(ctypes.byref(n)))
    return n.value


def version():
    return load().msc_version().decode()
