"""The lossless coding stage of edit records (Sec. 4.7 / 5.5: zstd after packing) and the
key-value record of floating edits, on CPU: both are host code in the library, so they run
without a GPU.  Records round-trip exactly; a mostly-zero q-map record codes far below its
raw size; damaged input is rejected."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2409_17346_gb300 import msc


@pytest.fixture(scope="module")
def lib():
    from paper_2409_17346_gb300 import build
    build.build()
    lib = msc.load()
    if lib.msc_coded_bound(16) == 0:
        pytest.skip("no zstd library on this machine")
    return msc


def test_code_decode_round_trip(lib):
    rng = np.random.default_rng(5)
    for rec in (np.zeros(0, np.uint8), np.zeros(1 << 16, np.uint8), rng.integers(0, 256, 5000).astype(np.uint8),
                np.repeat(rng.integers(0, 4, 4000), 17).astype(np.uint8)):
        for level in (1, 3, 19):
            coded = lib.code_record(rec, level)
            assert np.array_equal(lib.decode_record(coded), rec)


def test_mostly_zero_packed_record_codes_small(lib):
    """A q-map record of the shape the loop leaves (a few percent of vertices edited, the rest
    zero), packed by the oracle's packer, then coded: far below the packed size."""
    rng = np.random.default_rng(6)
    n = 200000
    q = np.zeros(n, np.uint8)
    hit = rng.random(n) < 0.03
    q[hit] = rng.integers(1, 7, hit.sum())
    lossless = rng.random(n) < 0.01
    q[lossless] = 0xFF
    vals = rng.standard_normal(int(lossless.sum())).astype(np.float32)
    packed = oracle.pack_edits(q, 6, vals)
    coded = lib.code_record(packed, 3)
    assert len(coded) < 0.6 * len(packed)
    assert np.array_equal(lib.decode_record(coded), packed)


def test_damaged_frames_are_rejected(lib):
    rec = np.arange(3000, dtype=np.uint8)
    coded = lib.code_record(rec, 3)
    bad = coded.copy()
    bad[:4] = 0
    with pytest.raises(msc.MscError) as e:
        lib.decode_record(bad)
    assert e.value.status == 1
    with pytest.raises(msc.MscError):
        lib.decode_record(coded[: len(coded) // 2])
    with pytest.raises(msc.MscError):
        lib.code_record(rec, 0)


def test_key_value_record_round_trip(lib):
    n = 1000
    idx = np.array([0, 3, 17, 999], np.uint64)
    val = np.float32([1.5, -0.0, 3e-38, -7.25])
    q = np.zeros(n, np.uint8)
    q[idx.astype(np.int64)] = 0xFF
    edits = dict(q_map=q, lossless_idx=idx, lossless_val=val)
    buf = lib.pack_edits_kv(edits)
    assert buf.size == 32 + 8 * len(idx)
    assert bytes(buf[:5]) == b"MSCE\x02"
    back = lib.unpack_edits_kv(buf, (n,))
    assert np.array_equal(back["q_map"].reshape(-1), q)
    assert np.array_equal(back["lossless_idx"].astype(np.uint64), idx)
    assert np.array_equal(back["lossless_val"].view(np.uint32), val.view(np.uint32))
    # quantised counts cannot become key-value pairs; damaged records are rejected
    q2 = q.copy()
    q2[5] = 2
    with pytest.raises(msc.MscError):
        lib.pack_edits_kv(dict(q_map=q2, lossless_idx=idx, lossless_val=val))
    bad = buf.copy()
    bad[32:36] = bad[36:40]                        # two equal vertex ids
    with pytest.raises(msc.MscError):
        lib.unpack_edits_kv(bad, (n,))
    with pytest.raises(msc.MscError):
        lib.unpack_edits_kv(buf[:-1], (n,))
