"""Batched and served fixes on the GPU: jobs that run concurrently on one device give the
same results as each job alone, and those results equal the CPU oracle's."""
import threading
import time

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


def _mixed_cases():
    """Uneven sizes and kinds, small enough for the oracle."""
    cases = [synth.config_case("grf3d", seed=40 + i, size=9 + 2 * i, rel=1e-2) for i in range(4)]
    cases += [synth.config_case("multiscale2d", seed=50 + i, size=(30 + 7 * i, 41 + 5 * i), rel=1e-2) for i in range(3)]
    cases += [synth.config_case("gauss2d", seed=60 + i) for i in range(2)]
    cases += [synth.config_case("kolmogorov3d", seed=70, size=13, rel=3e-3)]
    return cases


def _same(g1, ed1, g2, ed2):
    assert np.array_equal(np.asarray(g1).view(np.uint32), np.asarray(g2).view(np.uint32))
    assert (ed1["n_iters_c"], ed1["n_iters_s"], ed1["n_fallback_iters"]) == \
        (ed2["n_iters_c"], ed2["n_iters_s"], ed2["n_fallback_iters"])
    assert np.array_equal(ed1["q_map"], ed2["q_map"])


def _oracle_same(f, fh, xi, g, ed, tier=4):
    r = oracle.fix(f, fh, xi, tier=tier)
    assert r["status"] == 0
    assert np.array_equal(np.asarray(g).view(np.uint32), r["g"].view(np.uint32))
    assert (ed["n_iters_c"], ed["n_iters_s"]) == (r["n_c"], r["n_s"])


def test_batch_more_jobs_than_streams_matches_oracle(lib):
    cases = _mixed_cases()
    assert len(cases) > 8
    hs = [lib.Handle(c[0]) for c in cases]
    gs, eds = lib.fix_batch(hs, [c[1] for c in cases], [c[2] for c in cases], tier=4)
    for (f, fh, xi, _), g, ed in zip(cases, gs, eds):
        _oracle_same(f, fh, xi, g, ed)
    for h in hs:
        h.close()


def test_batch_device_buffers_on_caller_stream(lib):
    import torch
    cases = _mixed_cases()[:5]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        fhs = [torch.from_numpy(c[1]).cuda() for c in cases]
        gos = [torch.empty_like(x) for x in fhs]
    hs = [lib.Handle(c[0]) for c in cases]
    _, eds = lib.fix_batch(hs, fhs, [c[2] for c in cases], g_outs=gos, tier=4, stream=s.cuda_stream)
    for (f, fh, xi, _), h, g, ed in zip(cases, hs, gos, eds):
        g1, ed1 = lib.Handle(f).fix(fh, xi, tier=4)
        _same(g.cpu().numpy(), ed, g1, ed1)
        h.close()


def test_batch_rejects_shared_handles(lib):
    f, fh, xi, _ = synth.config_case("gauss2d")
    h = lib.Handle(f)
    with pytest.raises(lib.MscError, match="share a handle"):
        lib.fix_batch([h, h], [fh, fh], [xi, xi])
    h.close()


def test_server_results_equal_alone_and_oracle(lib):
    cases = _mixed_cases()
    alone = [lib.Handle(c[0]).fix(c[1], c[2], tier=4) for c in cases]
    with lib.Server(max_jobs=4, tier=4) as srv:
        tickets = [srv.submit(c[0], c[1], c[2]) for c in cases]
        done = [srv.wait(t) for t in tickets]
    slots = set()
    for (f, fh, xi, _), (g1, ed1), (g, ed, info) in zip(cases, alone, done):
        assert info["status"] == 0 and info["t_submit"] <= info["t_start"] <= info["t_end"]
        _same(g, ed, g1, ed1)
        _oracle_same(f, fh, xi, g, ed)
        slots.add(info["slot"])
    assert slots <= {0, 1, 2, 3}


def test_server_admission_respects_memory_budget(lib):
    cases = [synth.config_case("grf3d", seed=80 + i, size=20, rel=1e-2) for i in range(4)]
    need = lib.device_bytes(cases[0][0].shape)
    # room for two jobs at once, not three
    with lib.Server(max_jobs=4, mem_budget=2 * need + need // 2, tier=4) as srv:
        tickets = [srv.submit(c[0], c[1], c[2]) for c in cases]
        infos = [srv.wait(t)[2] for t in tickets]
    ev = sorted([(i["t_start"], 1) for i in infos] + [(i["t_end"], -1) for i in infos], key=lambda e: (e[0], e[1]))
    live = peak = 0
    for _, d in ev:
        live += d
        peak = max(peak, live)
    assert peak <= 2
    with lib.Server(max_jobs=2, mem_budget=need - 1) as srv:
        with pytest.raises(lib.MscError, match="budget"):
            srv.submit(cases[0][0], cases[0][1], cases[0][2])


def test_server_admits_jobs_arriving_while_others_run(lib):
    """Continuous batching: jobs submitted from another thread while earlier ones are on the
    device; every result equals the job alone."""
    big = synth.config_case("grf3d", seed=90, size=160, rel=1e-4)
    small = [synth.config_case("grf3d", seed=91 + i, size=12, rel=1e-2) for i in range(6)]
    alone_big = lib.Handle(big[0]).fix(big[1], big[2], tier=4)
    alone_small = [lib.Handle(c[0]).fix(c[1], c[2], tier=4) for c in small]
    results = {}
    with lib.Server(max_jobs=4, tier=4) as srv:
        tb = srv.submit(big[0], big[1], big[2])
        ts = []

        def arrive():
            for c in small:
                time.sleep(0.001)
                ts.append(srv.submit(c[0], c[1], c[2]))

        th = threading.Thread(target=arrive)
        th.start()
        th.join()
        results["big"] = srv.wait(tb)
        results["small"] = [srv.wait(t) for t in ts]
    _same(results["big"][0], results["big"][1], *alone_big)
    for (g, ed, _), (g1, ed1) in zip(results["small"], alone_small):
        _same(g, ed, g1, ed1)
    # the small jobs were admitted while the big one still ran
    bi = results["big"][2]
    assert any(info["t_start"] < bi["t_end"] for _, _, info in results["small"])
