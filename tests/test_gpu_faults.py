"""Failure paths made on the host, with no device fault: device allocations that fail at a
chosen point (prepare, fix, the server's admission), and serving jobs cancelled while
queued or running.  Each failing call must return its status cleanly, free what it had
allocated, and leave the library able to run the same fix again with the oracle's result."""
import time

import numpy as np
import pytest

import oracle
from paper_2409_17346_gb300 import synth

pytestmark = pytest.mark.gpu

OOM, CANCELLED = 2, 8


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2409_17346_gb300 import msc
    yield msc
    msc.inject_alloc_failures(0, 0)


def _fix_once(lib, f, fh, xi):
    h = lib.Handle(f)
    try:
        return h.fix(fh, xi, tier=4)
    finally:
        h.close()


@pytest.mark.parametrize("name,kw", [("kolmogorov3d", dict(size=12, rel=3e-3)), ("gauss2d", dict(seed=4))])
def test_every_allocation_failure_is_clean(lib, name, kw):
    """Fail the k-th device allocation of prepare + fix, for every k: the call reports
    MSC_ERR_OOM, the library's pool holds no more live memory than before, and the same fix
    afterwards equals the oracle's."""
    f, fh, xi, _ = synth.config_case(name, **kw)
    ref = oracle.fix(f, fh, xi, tier=4)
    _fix_once(lib, f, fh, xi)                 # warm: the pool holds its working set
    base = lib.pool_used_bytes()
    failures = 0
    for k in range(400):
        before = lib.inject_alloc_failures(k, 1)
        try:
            g, ed = _fix_once(lib, f, fh, xi)
            injected = lib.inject_alloc_failures(0, 0) - before
            assert injected == 0                   # k is past the last allocation
            assert np.array_equal(g.view(np.uint32), ref["g"].view(np.uint32))
            break
        except lib.MscError as e:
            lib.inject_alloc_failures(0, 0)
            assert e.status == OOM, e
            failures += 1
        assert lib.pool_used_bytes() == base
    else:
        pytest.fail("prepare + fix kept allocating")
    assert failures >= 5
    g, ed = _fix_once(lib, f, fh, xi)
    assert np.array_equal(g.view(np.uint32), ref["g"].view(np.uint32))
    assert (ed["n_iters_c"], ed["n_iters_s"]) == (ref["n_c"], ref["n_s"])


def test_server_admission_allocation_failure(lib):
    """The first admitted job's allocation fails: it ends with MSC_ERR_OOM and the jobs
    behind it still run and match the oracle."""
    cases = [synth.config_case("grf3d", seed=80 + i, size=10, rel=1e-2) for i in range(3)]
    with lib.Server(max_jobs=1) as srv:
        lib.inject_alloc_failures(0, 1)
        tickets = [srv.submit(f, fh, xi) for f, fh, xi, _ in cases]
        with pytest.raises(lib.MscError) as e:
            srv.wait(tickets[0])
        assert e.value.status == OOM
        lib.inject_alloc_failures(0, 0)
        for (f, fh, xi, _), t in zip(cases[1:], tickets[1:]):
            g, ed, info = srv.wait(t)
            ref = oracle.fix(f, fh, xi, tier=4)
            assert np.array_equal(g.view(np.uint32), ref["g"].view(np.uint32))


def test_server_cancel_queued_and_running(lib):
    """With one slot, a long job runs while others queue.  A cancelled queued job never
    starts; the running job, cancelled mid-loop, ends with MSC_ERR_CANCELLED unless it
    finished first; the jobs after them still match the oracle."""
    # floating edits take many more rounds than quantised ones, so the big job is still in
    # its fix loop when it is cancelled
    big = synth.config_case("kolmogorov3d", size=160, rel=1e-4)
    small = [synth.config_case("grf3d", seed=90 + i, size=10, rel=1e-2) for i in range(3)]
    with lib.Server(max_jobs=1, edit_mode=1) as srv:
        t_big = srv.submit(big[0], big[1], big[2])
        t_small = [srv.submit(f, fh, xi) for f, fh, xi, _ in small]
        srv.cancel(t_small[0])                 # queued behind the big job
        time.sleep(0.05)
        srv.cancel(t_big)                      # running (or already finished)
        with pytest.raises(lib.MscError) as e:
            srv.wait(t_small[0])
        assert e.value.status == CANCELLED
        try:
            srv.wait(t_big)
            big_status = 0
        except lib.MscError as e2:
            big_status = e2.status
        assert big_status in (0, CANCELLED)
        for (f, fh, xi, _), t in zip(small[1:], t_small[1:]):
            g, ed, info = srv.wait(t)
            ref = oracle.fix(f, fh, xi, tier=4, edit_mode=1)
            assert np.array_equal(g.view(np.uint32), ref["g"].view(np.uint32))
        with pytest.raises(lib.MscError):
            srv.cancel(t_small[1])             # already waited for: unknown ticket
    assert big_status == CANCELLED
