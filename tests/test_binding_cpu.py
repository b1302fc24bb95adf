"""The Python binding's handling of an edit record, on CPU with a record built by hand:
copies, zero-copy views that keep their owner alive exactly as long as some view exists,
and the trace conversion."""
import ctypes
import gc

import numpy as np
import pytest

from paper_2409_17346_gb300 import msc


class _Owner:
    freed = 0

    def __del__(self):
        _Owner.freed += 1


def _record(n, nl, nt):
    q = np.arange(n, dtype=np.uint8) % 7
    li = np.arange(nl, dtype=np.uint64) * 3
    lv = np.linspace(-1, 1, nl).astype(np.float32)
    tr = np.zeros(nt, dtype=msc._TRACE_DTYPE)
    tr["kind"] = np.arange(nt) % 2
    tr["t_us"] = np.arange(nt) * 10
    tr["n_targets"] = np.arange(nt) + 5
    tr["sum_targets"] = np.arange(nt) * 100
    e = msc.Edits()
    e.n_vertices, e.n_lossless, e.n_quant, e.n_trace = n, nl, n - nl, nt
    e.n_iters_c, e.n_iters_s = 3, 1
    e.q_map = q.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    e.lossless_idx = li.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    e.lossless_val = lv.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    e.trace = tr.ctypes.data_as(ctypes.POINTER(msc.IterRecord))
    return e, (q, li, lv, tr)


def test_iter_record_layout_matches_the_trace_dtype():
    assert ctypes.sizeof(msc.IterRecord) == msc._TRACE_DTYPE.itemsize == 40


def test_record_copies_and_trace():
    e, (q, li, lv, tr) = _record(24, 5, 4)
    out = msc._edits_to_py(e, (4, 6))
    assert out["q_map"].shape == (4, 6) and np.array_equal(out["q_map"].reshape(-1), q)
    assert np.array_equal(out["lossless_idx"], li) and np.array_equal(out["lossless_val"], lv)
    assert out["trace"].shape == (4, 5)
    assert np.array_equal(out["trace"][:, 0], tr["kind"]) and np.array_equal(out["trace"][:, 1], tr["n_targets"])
    assert np.array_equal(out["trace"][:, 3], tr["sum_targets"]) and np.array_equal(out["trace_t_us"], tr["t_us"])
    q[:] = 99                                  # copies do not follow the source
    assert not np.any(out["q_map"] == 99)


def test_record_views_keep_their_owner_until_the_last_view_goes():
    e, (q, li, lv, tr) = _record(16, 3, 0)
    _Owner.freed = 0
    out = msc._edits_to_py(e, (16,), _Owner())
    q[0] = 42                                  # views see the library's buffers
    assert out["q_map"][0] == 42
    qm, idx = out["q_map"], out["lossless_idx"]
    del out
    gc.collect()
    assert _Owner.freed == 0                   # two views still alive
    del qm
    gc.collect()
    assert _Owner.freed == 0
    del idx
    gc.collect()
    assert _Owner.freed == 1


def test_walk_limits_hook_checks_its_arguments_on_the_host():
    """msc_set_walk_limits validates on the host and touches no device: a per-warp stack
    above its 384 entries is rejected with MSC_ERR_INVALID_ARG; 0 restores the defaults."""
    msc.set_walk_limits(8, 4)
    msc.set_walk_limits(0, 0)
    with pytest.raises(msc.MscError) as e:
        msc.set_walk_limits(385, 0)
    assert e.value.status == 1
    msc.set_walk_limits(384, 1)
    msc.set_walk_limits(0, 0)
