"""Device logic of the CUDA path compiled for the host and checked on CPU, with no GPU (the
GPU parity tests check the kernels themselves):
  * the per-anchor gradient evaluator (eval_anchor and its compile-time cell tables) and the
    pair decoder, against the oracle's gradient;
  * the C-pass case logic (case_mask, case_apply, add_case), against the oracle's targeting
    pass: the same target set, restore set and number of cases;
  * the order-change filter of the edit round (order_changed, the window marks): every anchor
    whose code an edit changes is in the refresh set it builds;
  * the separatrix state of the S-pass (node_bits, the interleaved path walks, the
    saddle-saddle propagation, its incremental update, node_targets), against the oracle's
    S-pass: the same troublemaker targets and restores; likewise the terminal-mode walks of
    tier 3 (desc_walk, asc_walk);
  * the edit arithmetic of Eq. 2 (clamp_base, edit_apply), with the directed roundings taken
    from the host's IEEE rounding modes, against the oracle's values (its own TwoSum-based
    rounding) bit for bit."""
import ctypes
import os
import shutil
import subprocess
import zlib

import numpy as np
import pytest

import oracle
from paper_2409_17346_gb300 import synth

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
                               "-O2", "-Xcompiler", "-fPIC,-frounding-math", "-shared", "-o", tmp, SRC])
        os.replace(tmp, OUT)
    h = ctypes.CDLL(OUT)
    vp, i = ctypes.c_void_p, ctypes.c_int
    h.host_gradient_pairs.argtypes = [vp, i, i, i, vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
    h.host_cpass.argtypes = [vp, vp, vp, i, i, i, i, i, vp, vp, ctypes.POINTER(ctypes.c_uint64),
                             ctypes.POINTER(ctypes.c_uint64)]
    h.host_codes.argtypes = [vp, i, i, i, vp]
    h.host_dirty.argtypes = [vp, vp, vp, i, i, i, i, vp]
    h.host_spass.argtypes = [vp, vp, vp, vp, i, i, i, i, vp, vp, ctypes.POINTER(ctypes.c_uint64)]
    h.host_edit_sequence.argtypes = [vp, vp, ctypes.c_uint32, ctypes.c_float, i, i, vp, vp]
    h.host_spass_t3.argtypes = [vp, vp, vp, i, i, i, i, vp, vp]
    h.host_round.argtypes = [vp, vp, vp, vp, i, i, i, i, i, ctypes.c_float, i, i, ctypes.POINTER(ctypes.c_uint64),
                             ctypes.POINTER(ctypes.c_uint64)]
    return h


def _dims(shape):
    return shape[-1], shape[-2], (shape[0] if len(shape) == 3 else 1)


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


@pytest.mark.parametrize("shape", [(6, 7), (9, 5), (4, 5, 6), (3, 4, 3)])
@pytest.mark.parametrize("tier", [1, 2, 3, 4])
@pytest.mark.parametrize("fallback", [0, 1])
def test_device_cpass_matches_oracle_targets(lib, shape, tier, fallback):
    rng = np.random.default_rng(zlib.crc32(repr((shape, tier, fallback)).encode()))
    f = rng.standard_normal(shape).astype(np.float32)
    g = (f + rng.standard_normal(shape) * 0.6).astype(np.float32)
    # quantised states, floors and restores, so that live and stuck cases both occur
    st = rng.choice(np.array([0, 1, 3, 6, 0xF0, 0xF1], np.uint8), size=f.size, p=[.4, .2, .1, .1, .1, .1])
    st = np.ascontiguousarray(st, np.uint8)
    T = np.zeros(f.size, np.uint8)
    X = np.zeros(f.size, np.uint8)
    nc, nl = ctypes.c_uint64(), ctypes.c_uint64()
    lib.host_cpass(f.ctypes.data, g.ctypes.data, st.ctypes.data, *_dims(shape), tier, fallback, T.ctypes.data,
                   X.ctypes.data, ctypes.byref(nc), ctypes.byref(nl))
    cases, markX = oracle.targets(f, g, st, 0, tier, fallback)
    To = np.zeros(f.size, np.uint8)
    if len(cases):
        To[np.unique(cases[:, 0])] = 1
    assert nc.value == len(cases)
    assert np.array_equal(T, To)
    assert np.array_equal(X, (markX != 0).astype(np.uint8))
    live = [t for t in cases[:, 0] if st[t] not in (0xF0, 0xF1)]
    assert nl.value == len(live)


def test_order_change_filter_never_misses_a_changed_code(lib):
    """Random rounds: a fifth of the vertices lowered, by small or large amounts, so that
    moved vertices are often compared with other moved ones (each at its pre-round value).
    Every anchor whose code changed must be in the refresh set, both for the whole window of a
    vertex with any flipped pair and for the CUDA path's finer set (only the anchors whose
    windows hold both ends of a flipped pair); the sets must also leave many anchors out, the
    finer one more, or the filters would be doing nothing."""
    rng = np.random.default_rng(3)
    skipped = []
    skipped_pairwise = []
    for trial in range(200):
        shape = (tuple(int(s) for s in rng.integers(4, 9, 2)) if trial % 2 else tuple(int(s) for s in rng.integers(3, 7, 3)))
        a = rng.standard_normal(shape).astype(np.float32)
        moved = np.ascontiguousarray(rng.random(shape) < 0.2, np.uint8)
        step = np.where(rng.random(shape) < 0.7, rng.random(shape) * 0.05, rng.random(shape)).astype(np.float32)
        b = np.where(moved == 1, a - step, a).astype(np.float32)
        c0 = np.zeros(a.size, np.uint64)
        c1 = np.zeros(a.size, np.uint64)
        lib.host_codes(a.ctypes.data, *_dims(shape), c0.ctypes.data)
        lib.host_codes(b.ctypes.data, *_dims(shape), c1.ctypes.data)
        dirty = np.zeros(a.size, np.uint8)
        lib.host_dirty(a.ctypes.data, b.ctypes.data, moved.ctypes.data, *_dims(shape), 0, dirty.ctypes.data)
        assert not np.any((c0 != c1) & (dirty == 0)), trial
        skipped.append(1.0 - dirty.mean())
        pdirty = np.zeros(a.size, np.uint8)
        lib.host_dirty(a.ctypes.data, b.ctypes.data, moved.ctypes.data, *_dims(shape), 1, pdirty.ctypes.data)
        assert not np.any((c0 != c1) & (pdirty == 0)), trial
        assert not np.any((pdirty == 1) & (dirty == 0)), trial      # a subset of the whole windows
        skipped_pairwise.append(1.0 - pdirty.mean())
    assert np.mean(skipped) > 0.1
    assert np.mean(skipped_pairwise) > np.mean(skipped)


SPASS_CASES = [("gauss2d", dict(seed=9, size=(23, 41), rel=1e-2)), ("multiscale2d", dict(size=(40, 56), rel=1e-2)),
               ("grf3d", dict(size=9, rel=1e-2)), ("kolmogorov3d", dict(size=10, rel=3e-3)),
               ("grf3d", dict(size=13, rel=1e-2))]


@pytest.mark.parametrize("idx", range(len(SPASS_CASES)))
def test_device_separatrix_state_matches_oracle_spass(lib, idx):
    """Fields whose critical cells already equal f's (the oracle's tier-2 fix of two different
    base fields), so that the S-pass has troublemakers to find.  The state is built on one
    field and, in two of the three runs, updated to the other incrementally; either way its
    troublemakers must be the oracle's S-pass targets (the case counts differ by convention:
    the oracle counts paths, the state counts nodes)."""
    name, kw = SPASS_CASES[idx]
    f, fh, xi, _ = synth.config_case(name, **kw)
    fh2 = (f + np.random.default_rng(1).uniform(-xi, xi, f.shape)).astype(np.float32)
    r1, r2 = oracle.fix(f, fh, xi, tier=2), oracle.fix(f, fh2, xi, tier=2)
    for g1, g2, st in ((r1["g"], r1["g"], r1["state"]), (r1["g"], r2["g"], r2["state"]),
                       (r2["g"], r1["g"], r1["state"])):
        g1, g2 = np.ascontiguousarray(g1, np.float32), np.ascontiguousarray(g2, np.float32)
        st = np.ascontiguousarray(st, np.uint8).reshape(-1)
        T = np.zeros(f.size, np.uint8)
        X = np.zeros(f.size, np.uint8)
        nc = ctypes.c_uint64()
        assert lib.host_spass(f.ctypes.data, g1.ctypes.data, g2.ctypes.data, st.ctypes.data, *_dims(f.shape), 1,
                              T.ctypes.data, X.ctypes.data, ctypes.byref(nc)) == 0
        cases, markX = oracle.targets(f, g2, st, 1, 4, 1)
        To = np.zeros(f.size, np.uint8)
        if len(cases):
            To[np.unique(cases[:, 0])] = 1
        assert np.array_equal(T, To)
        assert np.array_equal(X, (markX != 0).astype(np.uint8))
        assert (nc.value > 0) == (len(cases) > 0)


@pytest.mark.parametrize("q_max,edit_mode", [(1, 0), (3, 0), (6, 0), (7, 0), (2, 1), (6, 1)])
def test_device_edit_arithmetic_matches_oracle(lib, q_max, edit_mode):
    """Every edit a vertex can take, from the re-clamped base through q_max quantised steps
    (every step down to f - xi for floating edits) to the floor, on values of three
    magnitudes, signed zeros, subnormals, bases 2 xi away (so the clamp matters) and bases
    equal to f."""
    rng = np.random.default_rng(100 + q_max)
    for xi in (1e-4, 1e-2, 0.5):
        n = 3000
        f = (rng.standard_normal(n) * rng.choice([1e-3, 1.0, 1e3], n)).astype(np.float32)
        f[:20], f[20:40], f[40:60] = np.float32(0.0), np.float32(-0.0), np.float32(1e-40)
        xi = float(np.float32(xi))
        fh = (f + rng.uniform(-2 * xi, 2 * xi, n)).astype(np.float32)
        fh[60:80] = f[60:80]
        # floating edits: no cap but the state byte's 0xEF steps, reached only where a step is
        # below half the float spacing of f and rounds back up to f - xi
        cap = 0xEF if edit_mode else q_max
        K = cap + 2
        g = np.zeros(n * K, np.float32)
        st = np.zeros(n * K, np.uint8)
        lib.host_edit_sequence(f.ctypes.data, fh.ctypes.data, n, xi, q_max, edit_mode, g.ctypes.data, st.ctypes.data)
        g, st = g.reshape(n, K), st.reshape(n, K)
        lb, ub, fc, qv = oracle.edit_values(f, fh, xi, q_max, n_steps=K)
        assert np.array_equal(g[:, 0].view(np.uint32), fc.view(np.uint32))
        was_floor = np.zeros(n, bool)
        for k in range(1, K):
            quant, floor = st[:, k] == k, st[:, k] == 0xF0
            assert np.all(quant | floor)
            if edit_mode:
                assert k < K - 1 or np.all(floor)              # past the cap every vertex is at its floor
            if k <= cap:
                assert np.array_equal(g[quant, k].view(np.uint32), qv[quant, k].view(np.uint32))
                assert np.all(qv[quant, k] >= lb[quant])
                first = floor & ~was_floor
                assert np.all(qv[first, k] < lb[first])       # the floor only when the step would pass it
            assert np.array_equal(g[floor, k].view(np.uint32), lb[floor].view(np.uint32))
            was_floor |= floor


@pytest.mark.parametrize("idx", range(len(SPASS_CASES)))
def test_device_tier3_walks_match_oracle_spass(lib, idx):
    name, kw = SPASS_CASES[idx]
    f, fh, xi, _ = synth.config_case(name, **kw)
    r = oracle.fix(f, fh, xi, tier=2)
    g = np.ascontiguousarray(r["g"], np.float32)
    st = np.ascontiguousarray(r["state"], np.uint8).reshape(-1)
    T = np.zeros(f.size, np.uint8)
    X = np.zeros(f.size, np.uint8)
    lib.host_spass_t3(f.ctypes.data, g.ctypes.data, st.ctypes.data, *_dims(f.shape), 1, T.ctypes.data, X.ctypes.data)
    cases, markX = oracle.targets(f, g, st, 1, 3, 1)
    To = np.zeros(f.size, np.uint8)
    if len(cases):
        To[np.unique(cases[:, 0])] = 1
    assert np.array_equal(T, To)
    assert np.array_equal(X, (markX != 0).astype(np.uint8))


ROUND_CASES = [("gauss2d", dict(seed=9, size=(23, 41), rel=1e-2)), ("multiscale2d", dict(size=(40, 56), rel=1e-2)),
               ("grf3d", dict(size=9, rel=1e-2)), ("kolmogorov3d", dict(size=10, rel=3e-3))]


@pytest.mark.parametrize("idx", range(len(ROUND_CASES)))
@pytest.mark.parametrize("fallback", [0, 1])
def test_fused_round_edits_equal_the_two_phase_round(lib, idx, fallback):
    """The persistent round kernel edits each target in its C-pass (reading the pre-round
    values from gprev, leaving the state for later), then applies the restores and the
    targets' states; the round graphs list all items first and edit them after.  From the
    same state, rounds of both forms give the same g (bit for bit), states, targets and
    restores, round after round (q_max 2 reaches the floor and stuck cases early)."""
    name, kw = ROUND_CASES[idx]
    f, fh, xi, _ = synth.config_case(name, **kw)
    f = np.ascontiguousarray(f, np.float32)
    fh = np.ascontiguousarray(fh, np.float32)
    q_max = 2
    n = f.size
    K = q_max + 2
    g0 = np.zeros(n * K, np.float32)
    s0 = np.zeros(n * K, np.uint8)
    lib.host_edit_sequence(f.ctypes.data, fh.ctypes.data, n, xi, q_max, 0, g0.ctypes.data, s0.ctypes.data)
    g = g0.reshape(n, K)[:, 0].copy()            # clamp(f_hat, [f - xi, f + xi])
    st = np.zeros(n, np.uint8)
    nt, nx = ctypes.c_uint64(0), ctypes.c_uint64(0)
    rounds = edited = 0
    for r in range(40):
        ga, sa = g.copy(), st.copy()
        gb, sb = g.copy(), st.copy()
        lib.host_round(f.ctypes.data, fh.ctypes.data, ga.ctypes.data, sa.ctypes.data, *_dims(f.shape), 4, fallback,
                       xi, q_max, 0, ctypes.byref(nt), ctypes.byref(nx))
        t0, x0 = nt.value, nx.value
        lib.host_round(f.ctypes.data, fh.ctypes.data, gb.ctypes.data, sb.ctypes.data, *_dims(f.shape), 4, fallback,
                       xi, q_max, 1, ctypes.byref(nt), ctypes.byref(nx))
        assert (nt.value, nx.value) == (t0, x0), r
        assert np.array_equal(ga.view(np.uint32), gb.view(np.uint32)), r
        assert np.array_equal(sa, sb), r
        if t0 + x0 == 0:
            break
        edited += int((ga != g).sum())
        rounds += 1
        g, st = ga, sa
    assert rounds >= 3 and edited > 0
