"""msc_critical_cells_static, the entry point that allocates no device memory, agrees
with msc_critical_cells (which allocates its own scratch) on caller-owned device
buffers, on two calls in a row, and leaves both torch's allocator and the library's
memory pool exactly as it found them."""
import numpy as np
import pytest

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


def _sorted(rows, dims):
    if len(rows):
        o = np.lexsort(rows.T[::-1])
        rows, dims = rows[o], dims[o]
    return rows, dims


def _static(lib, field, cap):
    import torch
    f = torch.from_numpy(field).cuda()
    rows = torch.full((max(cap, 1), 4), -7, dtype=torch.int64, device="cuda")
    dims = torch.full((max(cap, 1),), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    n = lib.critical_cells_static(f.data_ptr(), field.shape, rows.data_ptr(), dims.data_ptr(), cap, stream)
    m = min(n, cap)
    return n, rows[:m].cpu().numpy(), dims[:m].cpu().numpy(), rows[m:].cpu().numpy(), dims[m:].cpu().numpy()


CASES = [
    ("gauss2d", dict(size=None)),
    ("grf3d", dict(size=24)),
    ("kolmogorov3d", dict(size=32)),
]


@pytest.mark.parametrize("name,kw", CASES)
def test_static_matches_allocating_entry_point(lib, name, kw):
    f, f_hat, _, _ = synth.config_case(name, seed=3, **kw)
    for field in (f, f_hat):
        assert field.size <= lib.STATIC_MAX_VERTICES
        want_rows, want_dims = lib.critical_cells(field)
        for _ in range(2):
            n, rows, dims, tail_rows, tail_dims = _static(lib, field, len(want_rows) + 5)
            assert n == len(want_rows)
            rows, dims = _sorted(rows, dims)
            np.testing.assert_array_equal(rows, want_rows)
            np.testing.assert_array_equal(dims, want_dims)
            assert (tail_rows == -7).all() and (tail_dims == -7).all()


def test_static_truncates_at_cap(lib):
    f = synth.config_case("grf3d", seed=5, size=16)[0]
    want_rows, _ = lib.critical_cells(f)
    cap = len(want_rows) // 2
    n, rows, _, tail_rows, _ = _static(lib, f, cap)
    assert n == len(want_rows) and len(rows) == cap
    want = {tuple(r) for r in want_rows}
    assert all(tuple(r) in want for r in rows) and len({tuple(r) for r in rows}) == cap


def test_static_rejects_oversize_and_host_pointers(lib):
    import torch
    big = torch.zeros((1 << 10) + 1, 1 << 10, device="cuda")
    with pytest.raises(lib.MscError, match="static scratch limit"):
        lib.critical_cells_static(big.data_ptr(), tuple(big.shape), 0, 0, 0)
    host = np.zeros((8, 8), np.float32)
    with pytest.raises(lib.MscError, match="device pointers"):
        lib.critical_cells_static(host.ctypes.data, host.shape, 0, 0, 0)


def test_static_allocates_nothing(lib):
    """After a first call, further calls change neither torch's allocated bytes nor the
    bytes of the library's pool that live buffers hold."""
    import torch
    f = synth.config_case("grf3d", seed=7, size=20)[0]
    fd = torch.from_numpy(f).cuda()
    rows = torch.empty((4096, 4), dtype=torch.int64, device="cuda")
    dims = torch.empty((4096,), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    first = lib.critical_cells_static(fd.data_ptr(), f.shape, rows.data_ptr(), dims.data_ptr(), 4096, stream)
    torch.cuda.synchronize()
    torch_before = torch.cuda.memory_allocated()
    pool_before = lib.pool_used_bytes()
    for _ in range(3):
        n = lib.critical_cells_static(fd.data_ptr(), f.shape, rows.data_ptr(), dims.data_ptr(), 4096, stream)
        assert n == first
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == torch_before
    assert lib.pool_used_bytes() == pool_before
