"""The packed edit record on the GPU (msc_pack_edits / msc_unpack_edits) against the
oracle's packer, byte for byte, and the decompression side rebuilt from it bit-exactly."""
import numpy as np
import pytest

import oracle
from paper_2409_17346_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2409_17346_gb300 import msc
    return msc


CASES = [("gauss2d", {}, 6), ("multiscale2d", dict(size=(37, 45), rel=1e-2), 6),
         ("grf3d", dict(size=13, rel=1e-2), 3), ("kolmogorov3d", dict(size=11, rel=3e-3), 7),
         ("grf3d", dict(size=9, rel=1e-2), 1)]


@pytest.mark.parametrize("name,kw,q_max", CASES)
def test_pack_matches_oracle_and_rebuilds_g(lib, name, kw, q_max):
    f, fh, xi, tier = synth.config_case(name, **kw)
    g, ed = lib.Handle(f).fix(fh, xi, tier=tier, q_max=q_max)
    buf = lib.pack_edits(ed, q_max)
    want = oracle.pack_edits(ed["q_map"], q_max, ed["lossless_val"])
    assert buf.size == lib.packed_bytes(f.size, ed["n_lossless"], q_max) == want.size
    assert np.array_equal(buf, want)
    ed2, q2 = lib.unpack_edits(buf, f.shape)
    assert q2 == q_max and np.array_equal(ed2["q_map"], ed["q_map"])
    assert np.array_equal(ed2["lossless_idx"], ed["lossless_idx"])
    assert np.array_equal(ed2["lossless_val"].view(np.uint32), ed["lossless_val"].view(np.uint32))
    assert ed2["n_quant"] == ed["n_quant"] and ed2["n_lossless"] == ed["n_lossless"]
    g2 = lib.apply_edits(fh, xi, q2, ed2)
    assert np.array_equal(g2.view(np.uint32), g.view(np.uint32))


def test_unpack_oracle_record(lib):
    rng = np.random.default_rng(7)
    n = 12345
    qm = rng.integers(0, 7, n).astype(np.uint8)
    qm[rng.random(n) < 0.05] = 0xFF
    lv = rng.standard_normal(int((qm == 0xFF).sum())).astype(np.float32)
    buf = oracle.pack_edits(qm, 6, lv)
    ed, q = lib.unpack_edits(buf, (3, 4115))
    assert q == 6 and np.array_equal(ed["q_map"].reshape(-1), qm)
    assert np.array_equal(ed["lossless_idx"], np.nonzero(qm == 0xFF)[0].astype(np.uint64))


def test_pack_rejects_inconsistent_edits(lib):
    f, fh, xi, tier = synth.config_case("gauss2d")
    _, ed = lib.Handle(f).fix(fh, xi, tier=tier)
    bad = dict(ed)
    bad["q_map"] = ed["q_map"].copy()
    bad["q_map"].reshape(-1)[0] = 7          # above q_max = 6
    with pytest.raises(lib.MscError, match="above q_max"):
        lib.pack_edits(bad, 6)
    if ed["n_lossless"] >= 2:
        bad = dict(ed)
        bad["lossless_idx"] = ed["lossless_idx"][::-1].copy()
        with pytest.raises(lib.MscError, match="increasing order"):
            lib.pack_edits(bad, 6)
    buf = lib.pack_edits(ed, 6)
    with pytest.raises(lib.MscError):
        lib.unpack_edits(buf[:-1], f.shape)
    junk = buf.copy()
    junk[0] = ord("X")
    with pytest.raises(lib.MscError, match="header"):
        lib.unpack_edits(junk, f.shape)


def test_coded_records_rebuild_the_fix(lib):
    """Both stored forms of a fix go through the lossless coder and back: the quantised
    record (packed, then coded) and the floating-edit key-value record (coded); each rebuilds
    g bit-exactly through msc_apply_edits."""
    if lib.load().msc_coded_bound(16) == 0:
        pytest.skip("no zstd library on this machine")
    f, fh, xi, _ = synth.config_case("kolmogorov3d", size=24, rel=1e-3)
    g, ed = lib.Handle(f).fix(fh, xi, tier=4)
    packed = lib.pack_edits(ed, 6)
    coded = lib.code_record(packed, 3)
    back, q_max = lib.unpack_edits(lib.decode_record(coded), f.shape)
    assert q_max == 6
    assert np.array_equal(lib.apply_edits(fh, xi, 6, back).view(np.uint32), g.view(np.uint32))
    gf, edf = lib.Handle(f).fix(fh, xi, tier=4, edit_mode=1)
    kv = lib.pack_edits_kv(edf)
    backf = lib.unpack_edits_kv(lib.decode_record(lib.code_record(kv, 3)), f.shape)
    assert np.array_equal(lib.apply_edits(fh, xi, 6, backf).view(np.uint32), gf.view(np.uint32))
    ref = oracle.fix(f, fh, xi, tier=4, edit_mode=1)
    assert np.array_equal(gf.view(np.uint32), ref["g"].view(np.uint32))
