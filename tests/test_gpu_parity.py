"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer/index results (gradient pairs, critical cells, iteration counts, per-round target
digests, edit states) must be bit-exact; so must the corrected field g, because the method
is comparison work on fixed float32 values with correctly rounded edit arithmetic (no
tolerance applies anywhere)."""
import numpy as np
import pytest

import oracle
from paper_2409_17346_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2409_17346_gb300 import msc
    return msc


def _field(shape, kind, seed):
    rng = np.random.default_rng(seed)
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


SHAPES = [(2, 2), (2, 9), (9, 2), (37, 23), (64, 300), (2, 2, 2), (2, 3, 5), (13, 9, 11), (20, 17, 33),
          (18, 10, 67)]
KINDS = ["normal", "equal", "binary", "signed_zero", "levels"]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", KINDS)
def test_gradient_pairs_and_critical_cells(lib, shape, kind):
    a = _field(shape, kind, hash((shape, kind)) % 2**31)
    assert np.array_equal(lib.gradient_pairs(a), oracle.gradient_pairs(a))
    c1, d1 = lib.critical_cells(a)
    c2, d2 = oracle.critical_cells(a)
    assert np.array_equal(c1, c2) and np.array_equal(d1, d2)


def test_gradient_on_workload_fields(lib):
    for name, kw in (("gauss2d", {}), ("multiscale2d", dict(size=(90, 170))), ("grf3d", dict(size=24)),
                     ("kolmogorov3d", dict(size=24))):
        f, fh, _, _ = synth.config_case(name, **kw)
        for a in (f, fh):
            assert np.array_equal(lib.gradient_pairs(a), oracle.gradient_pairs(a))


FIX_CASES = [
    ("gauss2d", {}),                                       # the 64x64 workload itself
    ("gauss2d", dict(seed=9, size=(23, 41), rel=1e-2)),
    ("multiscale2d", dict(size=(40, 56), rel=1e-2)),
    ("multiscale2d", dict(size=(61, 130), rel=3e-3)),
    ("grf3d", dict(size=9, rel=1e-2)),
    ("grf3d", dict(size=13, rel=1e-2)),
    ("kolmogorov3d", dict(size=10, rel=3e-3)),
    ("kolmogorov3d", dict(size=16, rel=1e-3)),
]


def _check_fix(lib, f, fh, xi, tier, q_max=6, exact_fallback=1, small_round=0, edit_mode=0):
    ref = oracle.fix(f, fh, xi, tier=tier, q_max=q_max, exact_fallback=exact_fallback, edit_mode=edit_mode)
    assert ref["status"] == 0
    h = lib.Handle(f)
    g, ed = h.fix(fh, xi, tier=tier, q_max=q_max, exact_fallback=exact_fallback, record_trace=True,
                  small_round=small_round, edit_mode=edit_mode)
    assert np.array_equal(g.view(np.uint32), ref["g"].view(np.uint32))
    assert (ed["n_iters_c"], ed["n_iters_s"]) == (ref["n_c"], ref["n_s"])
    assert ed["n_fallback_iters"] == ref["n_exact_iters"]
    assert np.array_equal(ed["trace"], ref["trace"][:, :5])
    qm, li, lv = oracle.edits_from_state(f, fh, xi, ref["state"], ref["g"], edit_mode=edit_mode)
    assert np.array_equal(ed["q_map"].reshape(-1), qm)
    assert np.array_equal(ed["lossless_idx"].astype(np.int64), li)
    assert np.array_equal(ed["lossless_val"].view(np.uint32), lv.view(np.uint32))
    rep = h.verify(g, xi)
    assert rep["passed_tier"][tier - 1]
    assert all(rep["passed_tier"][:tier])
    h.close()
    return g, ed


@pytest.mark.parametrize("idx", range(len(FIX_CASES)))
@pytest.mark.parametrize("tier", [1, 2, 3, 4])
def test_fix_loop_matches_oracle(lib, idx, tier):
    name, kw = FIX_CASES[idx]
    f, fh, xi, _ = synth.config_case(name, **kw)
    _check_fix(lib, f, fh, xi, tier)


@pytest.mark.parametrize("idx", [0, 3, 7])
@pytest.mark.parametrize("tier", [2, 4])
def test_fix_loop_rounds_as_graph_nodes(lib, idx, tier):
    """Every round as captured graph nodes (the C-pass that marks T bits, then k_tlist),
    none in the persistent round kernel: the same result, round by round."""
    name, kw = FIX_CASES[idx]
    f, fh, xi, _ = synth.config_case(name, **kw)
    _check_fix(lib, f, fh, xi, tier, small_round=1)


@pytest.mark.parametrize("idx", [1, 3, 5, 7])
def test_fix_loop_without_cluster_rounds(lib, idx):
    """With the cluster form off, every small round runs in the full-grid persistent kernel:
    the same result, round by round."""
    name, kw = FIX_CASES[idx]
    f, fh, xi, _ = synth.config_case(name, **kw)
    ref = oracle.fix(f, fh, xi, tier=4)
    h = lib.Handle(f)
    g, ed = h.fix(fh, xi, tier=4, record_trace=True, cluster_round=1)
    st = h.stats()
    h.close()
    assert st["rounds"]["cluster_launches"] == 0
    assert np.array_equal(g.view(np.uint32), ref["g"].view(np.uint32))
    assert np.array_equal(ed["trace"], ref["trace"][:, :5])


def test_tiny_rounds_run_in_one_cluster(lib):
    """By default the rounds that follow one editing fewer than 1024 vertices run in the
    cluster form of the round kernel; a large case moves between the graph rounds, the
    full-grid kernel and the cluster form, and still equals the oracle round by round."""
    name, kw, tier, _ = LARGE_CASES[0]
    f, fh, xi, _ = synth.config_case(name, **kw)
    ref = oracle.fix(f, fh, xi, tier=tier)
    h = lib.Handle(f)
    g, ed = h.fix(fh, xi, tier=tier, record_trace=True)
    st = h.stats()
    h.close()
    assert st["rounds"]["cluster_launches"] > 0 and st["rounds"]["cluster_rounds"] > ed["n_iters_c"] // 2
    assert np.array_equal(g.view(np.uint32), ref["g"].view(np.uint32))
    assert np.array_equal(ed["trace"], ref["trace"][:, :5])


def test_small_rounds_run_in_the_round_kernel(lib):
    """With the default threshold the rounds after the first run in the persistent round
    kernel (this case edits fewer than 8192 vertices per round)."""
    name, kw = FIX_CASES[3]
    f, fh, xi, _ = synth.config_case(name, **kw)
    ref = oracle.fix(f, fh, xi, tier=4)
    h = lib.Handle(f)
    g, ed = h.fix(fh, xi, tier=4, record_trace=True)
    st = h.stats()
    h.close()
    assert np.array_equal(g.view(np.uint32), ref["g"].view(np.uint32))
    assert np.array_equal(ed["trace"], ref["trace"][:, :5])
    assert st["rounds"]["launches"] > 0
    assert st["rounds"]["items"] >= ed["n_iters_c"] // 2


# Larger cases, at the default round threshold: their first rounds edit 8192 vertices or
# more, so the loop takes the captured-graph rounds and then hands over to the persistent
# round kernel by itself; grids span many tiles, multi-wave launches and many listed
# 1024-anchor C-blocks, and separatrices cross many tiles.
LARGE_CASES = [
    ("kolmogorov3d", dict(size=64, rel=1e-4), 4, True),
    ("kolmogorov3d", dict(size=64, rel=1e-3), 4, True),
    ("kolmogorov3d", dict(size=48, rel=1e-3), 3, False),
    ("multiscale2d", dict(size=(512, 1024), rel=1e-3), 3, True),
    ("multiscale2d", dict(size=(512, 1024), rel=1e-2), 4, True),
]


@pytest.mark.parametrize("idx", range(len(LARGE_CASES)))
def test_fix_loop_matches_oracle_large(lib, idx):
    name, kw, tier, big_rounds = LARGE_CASES[idx]
    f, fh, xi, _ = synth.config_case(name, **kw)
    g, ed = _check_fix(lib, f, fh, xi, tier)
    tr = ed["trace"]
    if big_rounds:
        assert int((tr[:, 1] + tr[:, 2] >= 8192).sum()) >= 3
    assert ed["n_iters_c"] > 100


@pytest.mark.parametrize("limits", [(2, 2), (8, 4), (32, 16)])
@pytest.mark.parametrize("idx", [5, 7])
def test_saddle_walk_spill_paths_match_oracle(lib, idx, limits):
    """Tier 4 in 3D with the saddle-saddle walk's per-warp stack and per-thread step limit
    lowered, so that the first build and the updates spill most of their pending triangles
    to the queue that the converged spill kernel drains: the same result, round by round."""
    name, kw = FIX_CASES[idx]
    f, fh, xi, _ = synth.config_case(name, **kw)
    lib.set_walk_limits(*limits)
    try:
        _check_fix(lib, f, fh, xi, 4)
        _check_fix(lib, f, fh, xi, 4, small_round=1)
    finally:
        lib.set_walk_limits(0, 0)


def test_saddle_walk_spill_paths_large(lib):
    """The same on a 48^3 field with a 16-entry stack and 8-step walks."""
    f, fh, xi, _ = synth.config_case("kolmogorov3d", size=48, rel=1e-3)
    lib.set_walk_limits(16, 8)
    try:
        _check_fix(lib, f, fh, xi, 4)
    finally:
        lib.set_walk_limits(0, 0)


def test_walk_limits_reject_a_stack_above_its_size(lib):
    with pytest.raises(lib.MscError):
        lib.set_walk_limits(385, 0)
    lib.set_walk_limits(0, 0)


@pytest.mark.parametrize("idx", [0, 3, 5, 7])
@pytest.mark.parametrize("q_max", [2, 6])
def test_floating_edit_mode_matches_oracle(lib, idx, q_max):
    """Floating edits (no cap on the step count; every edit stored as an exact value): the
    same bit-exact agreement with the oracle, round by round."""
    name, kw = FIX_CASES[idx]
    f, fh, xi, _ = synth.config_case(name, **kw)
    g, ed = _check_fix(lib, f, fh, xi, 4, q_max=q_max, edit_mode=1)
    assert ed["n_quant"] == 0 and set(np.unique(ed["q_map"])) <= {0, 0xFF}
    g2 = lib.apply_edits(fh, xi, q_max, ed)
    assert np.array_equal(g2.view(np.uint32), g.view(np.uint32))


def test_floating_edit_mode_rejects_q_max_7(lib):
    f, fh, xi, _ = synth.config_case("gauss2d", seed=4, size=(20, 20), rel=1e-2)
    with pytest.raises(lib.MscError) as e:
        lib.Handle(f).fix(fh, xi, q_max=7, edit_mode=1)
    assert e.value.status == 1


def test_every_tile_shape_matches_oracle(lib):
    """The dense 3D gradient gives the oracle's result with every instantiated tile shape (the
    grid spans several tiles, slabs and a ragged edge in each direction), and the autotuner
    keeps one of them."""
    f, fh, xi, _ = synth.config_case("kolmogorov3d", seed=12, size=37, rel=3e-3)
    f = np.ascontiguousarray(f[:, :29, :])
    fh = np.ascontiguousarray(fh[:, :29, :])
    ref = oracle.fix(f, fh, xi, tier=4)
    pairs = oracle.gradient_pairs(f)
    shapes = lib.tile_report(f.shape)["shapes"]
    assert len(shapes) >= 4
    for tile in shapes:
        h = lib.Handle(f, opts=lib.options(tile=tile))
        g, ed = h.fix(fh, xi, tier=4, tile=tile)
        h.close()
        assert np.array_equal(g.view(np.uint32), ref["g"].view(np.uint32)), tile
        assert (ed["n_iters_c"], ed["n_iters_s"]) == (ref["n_c"], ref["n_s"]), tile
    g, _ = lib.Handle(f).fix(fh, xi, tier=4)
    rep = lib.tile_report(f.shape)
    assert rep["chosen"] in shapes and all(m > 0 for m in rep["ms"])
    assert np.array_equal(g.view(np.uint32), ref["g"].view(np.uint32))
    assert np.array_equal(lib.gradient_pairs(f), pairs)
    with pytest.raises(lib.MscError):
        lib.Handle(f, opts=lib.options(tile=(32, 5, 16)))


@pytest.mark.parametrize("q_max", [1, 3, 7])
def test_fix_q_max_range(lib, q_max):
    f, fh, xi, _ = synth.config_case("gauss2d", seed=4, size=(30, 33), rel=1e-2)
    _check_fix(lib, f, fh, xi, 4, q_max=q_max)


def test_device_and_host_pointers_agree(lib):
    import torch
    f, fh, xi, tier = synth.config_case("grf3d", size=12, rel=1e-2)
    h = lib.Handle(torch.from_numpy(f).cuda())
    gd = torch.empty(f.shape, dtype=torch.float32, device="cuda")
    h.fix(torch.from_numpy(fh).cuda(), xi, g_out=gd, tier=4)
    g_host, _ = lib.Handle(f).fix(fh, xi, tier=4)
    assert np.array_equal(gd.cpu().numpy().view(np.uint32), g_host.view(np.uint32))


def test_apply_edits_rebuilds_g_bit_exactly(lib):
    import torch
    for name, kw in (("multiscale2d", dict(size=(50, 70), rel=1e-2)), ("kolmogorov3d", dict(size=12, rel=3e-3))):
        f, fh, xi, _ = synth.config_case(name, **kw)
        g, ed = lib.Handle(f).fix(fh, xi, tier=4)
        g2 = lib.apply_edits(fh, xi, 6, ed)
        assert np.array_equal(g2.view(np.uint32), g.view(np.uint32))
        g3 = torch.empty(f.shape, dtype=torch.float32, device="cuda")
        lib.apply_edits(torch.from_numpy(fh).cuda(), xi, 6, ed, g_out=g3)
        assert np.array_equal(g3.cpu().numpy().view(np.uint32), g.view(np.uint32))
        # the oracle's decompression side reads the same stored edits
        g4 = oracle.apply_edits(fh, xi, 6, ed["q_map"].reshape(-1), ed["lossless_idx"].astype(np.int64), ed["lossless_val"])
        assert np.array_equal(g4.view(np.uint32), g.view(np.uint32))


def test_verify_matches_oracle_report(lib):
    """Every count of msc_verify equals the oracle's, including the number of 2-saddles
    whose saddle-saddle connectors differ."""
    saddle_counts = []
    for name, kw in (("gauss2d", {}), ("multiscale2d", dict(size=(45, 64), rel=1e-2)),
                     ("grf3d", dict(size=11, rel=1e-2)), ("grf3d", dict(seed=8, size=14, rel=3e-3)),
                     ("kolmogorov3d", dict(size=16, rel=1e-3))):
        f, fh, xi, _ = synth.config_case(name, **kw)
        h = lib.Handle(f)
        for tier in (2, 3):
            g = oracle.fix(f, fh, xi, tier=tier)["g"]
            for field in (np.clip(fh, f - xi, f + xi).astype(np.float32), g):
                r = h.verify(field, xi)
                o = oracle.verify(f, field)
                assert r["fp"] == [o["fp%d" % d] for d in range(4)]
                assert r["fn"] == [o["fn%d" % d] for d in range(4)]
                assert r["sep_mismatch"][:2] == [o["sep_desc"], o["sep_asc"]]
                assert r["term_mismatch"] == [o["term_desc"], o["term_asc"]]
                assert r["sep_mismatch"][2] == o["sep_saddle"]
                assert abs(r["max_abs_err"] - o["max_abs_err"]) == 0.0
                saddle_counts.append(o["sep_saddle"])
    assert max(saddle_counts) > 0


def test_edge_cases(lib):
    # no edits needed: f_hat == f
    f, _, xi, _ = synth.config_case("grf3d", size=9, rel=1e-2)
    g, ed = lib.Handle(f).fix(f, xi)
    assert np.array_equal(g, f) and ed["n_iters_c"] == 0 and ed["n_iters_s"] == 0 and ed["n_lossless"] == 0
    # constant original field (every tie broken by index), noisy base
    c = np.zeros((12, 15), np.float32)
    _check_fix(lib, c, (c + np.random.default_rng(1).uniform(-0.1, 0.1, c.shape)).astype(np.float32), 0.1, 4)
    # smallest grids
    for shape in ((2, 2), (2, 7), (2, 2, 2), (3, 2, 2)):
        f = _field(shape, "normal", 3)
        fh = (f + np.random.default_rng(2).uniform(-0.5, 0.5, shape)).astype(np.float32)
        _check_fix(lib, f, fh, 0.5, 4)


def test_float_tie_stall_and_fallback(lib):
    a = np.float32(-1.0 + 2.0 ** -24)
    b = np.float32(-1.0 + 2.0 ** -23)
    xi = float(np.float32(2.0 ** -23))
    f = np.float32([[b, a], [10, 11]])
    fh = np.float32([[-1.0, a + 2 ** -24], [10, 11]])
    _check_fix(lib, f, fh, xi, 4)
    with pytest.raises(lib.MscError) as e:
        lib.Handle(f).fix(fh, xi, exact_fallback=0)
    assert e.value.status == 6


def test_invalid_arguments(lib):
    f = np.zeros((4, 5), np.float32)
    bad = f.copy()
    bad[2, 2] = np.nan
    with pytest.raises(lib.MscError) as e:
        lib.Handle(bad)
    assert e.value.status == 1
    h = lib.Handle(f)
    for kw, xi, fh in ((dict(), 0.1, bad), (dict(), 0.0, f), (dict(q_max=8), 0.1, f), (dict(tier=5), 0.1, f)):
        with pytest.raises(lib.MscError) as e:
            h.fix(fh, xi, **kw)
        assert e.value.status == 1
    with pytest.raises(lib.MscError) as e:
        lib.Handle(np.zeros((1, 5), np.float32))
    assert e.value.status == 1
    f2, fh2, xi2, _ = synth.config_case("gauss2d")
    with pytest.raises(lib.MscError) as e:
        lib.Handle(f2).fix(fh2, xi2, max_iters=1)
    assert e.value.status == 4


def test_handle_reuse_after_error_and_repeat(lib):
    """A handle stays correct after a call that stopped early and across repeated fixes."""
    f, fh, xi, _ = synth.config_case("kolmogorov3d", size=14, rel=1e-3)
    h = lib.Handle(f)
    with pytest.raises(lib.MscError):
        h.fix(fh, xi, tier=4, max_iters=3)
    ref = oracle.fix(f, fh, xi, tier=4)
    for _ in range(2):
        g, ed = h.fix(fh, xi, tier=4)
        assert np.array_equal(g.view(np.uint32), ref["g"].view(np.uint32))
        assert (ed["n_iters_c"], ed["n_iters_s"]) == (ref["n_c"], ref["n_s"])
    f2, fh2, xi2, _ = synth.config_case("kolmogorov3d", seed=11, size=14, rel=1e-3)
    ref2 = oracle.fix(f, fh2, xi2, tier=4)
    g2, _ = h.fix(fh2, xi2, tier=4)
    assert np.array_equal(g2.view(np.uint32), ref2["g"].view(np.uint32))


def test_batch_equals_single(lib):
    cases = [synth.config_case("grf3d", seed=30 + i, size=11, rel=1e-2) for i in range(3)]
    cases += [synth.config_case("gauss2d", seed=5)]
    hs = [lib.Handle(c[0]) for c in cases]
    gs, eds = lib.fix_batch(hs, [c[1] for c in cases], [c[2] for c in cases], tier=4)
    for (f, fh, xi, _), g, ed in zip(cases, gs, eds):
        g1, ed1 = lib.Handle(f).fix(fh, xi, tier=4)
        assert np.array_equal(g.view(np.uint32), g1.view(np.uint32))
        assert (ed["n_iters_c"], ed["n_iters_s"]) == (ed1["n_iters_c"], ed1["n_iters_s"])


# ------------------------------------------------------------------------------------
# full-size workloads: properties that hold at any size, plus oracle checks on samples
# ------------------------------------------------------------------------------------

def _window_crit(field, box):
    """critical cells of a sub-block, keeping only cells two vertices inside it"""
    (z0, z1), (y0, y1), (x0, x1) = box
    sub = np.ascontiguousarray(field[z0:z1, y0:y1, x0:x1] if field.ndim == 3 else field[y0:y1, x0:x1])
    cells, dims = oracle.critical_cells(sub)
    shp = sub.shape
    keep = []
    for c, d in zip(cells, dims):
        ok = True
        for v in c[c >= 0]:
            idx = np.unravel_index(v, shp)
            ok = ok and all(2 <= i < s - 2 for i, s in zip(idx, shp))
        if ok:
            keep.append((tuple(c), int(d)))
    return sorted(keep)


def _full_size_check(lib, f, fh, xi, tier, n_windows=6, win=14):
    import torch
    fd, fhd = torch.from_numpy(f).cuda(), torch.from_numpy(fh).cuda()
    gd = torch.empty_like(fd)
    h = lib.Handle(fd)
    _, ed = h.fix(fhd, xi, g_out=gd, tier=tier)
    rep = h.verify(gd, xi)
    assert rep["passed_tier"][tier - 1], rep
    g = gd.cpu().numpy()
    # bound, exactly (float differences of nearby values are exact in float64)
    assert np.all(np.abs(g.astype(np.float64) - f.astype(np.float64)) <= xi)
    # every stored state is one of Eq. 2's values (or a restore), recomputed by the oracle
    lb, ub, fc, qv = oracle.edit_values(f.reshape(-1), fh.reshape(-1), xi, 6)
    qm = ed["q_map"].reshape(-1)
    quant = qm != 0xFF
    assert np.array_equal(g.reshape(-1)[quant].view(np.uint32),
                          qv[np.nonzero(quant)[0], qm[quant]].view(np.uint32))
    # decompression side rebuilds g
    g2 = lib.apply_edits(fh, xi, 6, ed)
    assert np.array_equal(g2.view(np.uint32), g.view(np.uint32))
    # sampled windows: the oracle sees the same critical cells in g as in f
    rng = np.random.default_rng(7)
    for _ in range(n_windows):
        box = [(0, 1)] if f.ndim == 2 else []
        for s in f.shape:
            o = int(rng.integers(0, s - win + 1))
            box.append((o, o + win))
        if f.ndim == 2:
            box = [(0, 1)] + box[1:]
        assert _window_crit(g, box if f.ndim == 3 else box) == _window_crit(f, box if f.ndim == 3 else box)
    return ed


def test_full_size_multiscale_2d(lib):
    f, fh, xi, tier = synth.config_case("multiscale2d")
    _full_size_check(lib, f, fh, xi, tier)


def test_full_size_grf_256(lib):
    f, fh, xi, tier = synth.config_case("grf3d")
    _full_size_check(lib, f, fh, xi, tier, n_windows=4, win=12)


def test_full_size_kolmogorov_512(lib):
    f, fh, xi, tier = synth.config_case("kolmogorov3d")
    _full_size_check(lib, f, fh, xi, tier, n_windows=4, win=12)


def test_fix_after_releasing_cached_memory(lib):
    """Handles freed into the library's pool, the pool trimmed, then the same fix again."""
    f, fh, xi, _ = synth.config_case("grf3d", seed=7, size=20, rel=1e-3)
    g1, e1 = lib.Handle(f).fix(fh, xi, tier=4)
    lib.release_cached_memory()
    g2, e2 = lib.Handle(f).fix(fh, xi, tier=4)
    assert np.array_equal(g1.view(np.uint32), g2.view(np.uint32))
    assert (e1["n_iters_c"], e1["n_iters_s"]) == (e2["n_iters_c"], e2["n_iters_s"])
