"""The q_max sweep and the extreme-noise stress case on the GPU, each against the oracle:
bit-exact g, iteration counts, per-round digests and stored edits."""
import numpy as np
import pytest

from paper_2409_17346_gb300 import synth
from test_gpu_parity import _check_fix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2409_17346_gb300 import msc
    return msc


@pytest.mark.parametrize("q_max", [2, 3, 4, 5, 6, 7])
def test_q_max_sweep_matches_oracle(lib, q_max):
    f, fh, xi, _ = synth.config_case("multiscale2d", seed=11, size=(48, 60), rel=1e-2)
    _check_fix(lib, f, fh, xi, 4, q_max=q_max)
    f, fh, xi, _ = synth.config_case("grf3d", seed=12, size=12, rel=1e-2)
    _check_fix(lib, f, fh, xi, 4, q_max=q_max)


@pytest.mark.parametrize("n", [16, 33, 48])
@pytest.mark.parametrize("tier", [1, 2, 3, 4])
def test_extreme_noise_matches_oracle(lib, n, tier):
    f, fh, xi = synth.extreme_noise_2d(n, seed=n)
    assert np.all(np.abs(f.astype(np.float64) - fh) <= xi)
    _check_fix(lib, f, fh, xi, tier)


def test_extreme_noise_large_properties(lib):
    """At sizes beyond the oracle: the MSC is preserved, the bound holds, edits only lower."""
    f, fh, xi = synth.extreme_noise_2d(1024, seed=3)
    h = lib.Handle(f)
    g, ed = h.fix(fh, xi, tier=4)
    rep = h.verify(g, xi)
    assert rep["passed"] and rep["max_abs_err"] <= xi
    assert np.all(g <= np.maximum(fh, f))          # lowered from the base, or restored to f
    assert ed["n_quant"] + ed["n_lossless"] > 0.1 * f.size
    h.close()
