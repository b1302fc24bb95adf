"""The bounded grid barrier of the persistent round kernel: a wait for a block that never
arrives gives up after its limit, reports MSC_ERR_DEVICE_TIMEOUT, and leaves the device
usable.  (No fault, trap or endless loop: the wait has a limit by construction.)"""
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


def test_barrier_wait_gives_up_and_device_stays_usable(lib):
    t0 = time.perf_counter()
    status = lib.selftest_barrier(200)
    dt = time.perf_counter() - t0
    assert status == 5                      # MSC_ERR_DEVICE_TIMEOUT
    assert 0.15 < dt < 5.0
    # a fix whose small rounds run in the persistent kernel still matches the oracle
    f, fh, xi, _ = synth.config_case("gauss2d", seed=9, size=(23, 41), rel=1e-2)
    g, ed = lib.Handle(f).fix(fh, xi, tier=4)
    ref = oracle.fix(f, fh, xi, tier=4)
    assert np.array_equal(g.view(np.uint32), ref["g"].view(np.uint32))
    assert (ed["n_iters_c"], ed["n_iters_s"]) == (ref["n_c"], ref["n_s"])


def test_barrier_selftest_rejects_bad_limits(lib):
    assert lib.selftest_barrier(0) == 1
    assert lib.selftest_barrier(5000) == 1
