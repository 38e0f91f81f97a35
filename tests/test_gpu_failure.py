"""Failure detection without a GPU fault: bounded device waits return an error status.

A cooperative launch in which one block never arrives at the grid barrier makes every other
block's wait run out after a short limit; the host reads SF_ERR_TIMEOUT and the context stays
usable (a normal launch and a sketch update succeed afterwards).  Host-side failures (bad
arguments, underflow, bad key ids) are covered in the parity and ABI tests."""
import pytest

pytestmark = pytest.mark.gpu


def test_barrier_wait_times_out_and_the_context_survives(sf):
    import torch
    L = sf.load_bench()
    scratch = torch.zeros(64, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert L.sf_bench_wait_timeout(scratch.data_ptr(), 0, 20_000_000, st) == sf.SF_OK
    assert L.sf_bench_wait_timeout(scratch.data_ptr(), 1, 20_000_000, st) == sf.SF_ERR_TIMEOUT
    assert L.sf_bench_wait_timeout(scratch.data_ptr(), 5, 20_000_000, st) == sf.SF_ERR_TIMEOUT
    # the context is still usable
    assert L.sf_bench_grid_barrier(scratch.data_ptr(), 10, st) == sf.SF_OK
    g = sf.Sketch(4, 1024, 16, 4, 1, 256)
    g.insert(torch.arange(1000, dtype=torch.int32, device="cuda"))
    assert g.sync_status() == sf.SF_OK
    assert int((g.fat.view(4, -1).to(torch.int64).sum(dim=1) == 1000).sum()) == 4


def test_wait_limit_is_bounded_by_the_api(sf):
    import torch
    L = sf.load_bench()
    scratch = torch.zeros(64, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert L.sf_bench_wait_timeout(scratch.data_ptr(), 1, 5_000_000_000, st) == sf.SF_ERR_INVALID
