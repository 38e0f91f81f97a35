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


def test_timeout_status_rezeroes_shared_dictionaries_and_the_arena(sf):
    """A grid wait that gave up latches the timeout bit in the error word (the first control word
    of the scratch) and may leave dictionary entries claimed.  Here the host writes that bit and
    fills the dictionaries with stale claim words, standing in for such a launch (no kernel is made
    to time out): sf_sync returns SF_ERR_TIMEOUT and zeroes the scratch and the dictionary given by
    sf_set_dictionary, sf_batch_sync zeroes the batch's dictionary arena, and the next updates
    equal sketches that never saw the failure.  The stale words (0x11111111) carry no fingerprint a
    key can have, so a dictionary left dirty would show up as wrong counters or a full-dictionary
    error, never as a re-read of a key."""
    import torch
    import workloads as wl
    ins, dels, _ = wl.flows_with_deletes(60_000, 8_000, 1.0, 0.1, seed=91, device="cuda")
    need = sf.dictionary_bytes(4, 3001, 16, 13, 5, 4096)
    a = sf.Sketch(4, 3001, 16, 13, 5, 4096)
    b = sf.Sketch(4, 3001, 16, 13, 5, 4096, shared_dict=True)
    d = torch.empty(need, dtype=torch.uint8, device="cuda")
    b.set_dictionary(d)
    torch.cuda.synchronize()
    d.fill_(0x11)
    b.scratch[0] = 2
    torch.cuda.synchronize()
    assert b.sync_status() == sf.SF_ERR_TIMEOUT
    assert int(torch.count_nonzero(d)) == 0 and int(torch.count_nonzero(b.scratch[:64])) == 0
    assert b.sync_status() == sf.SF_OK
    for s in (a, b):
        s.insert(ins)
        s.delete(dels)
    assert a.sync_status() == sf.SF_OK and b.sync_status() == sf.SF_OK
    assert torch.equal(a.fat, b.fat) and torch.equal(a.slim, b.slim)

    c = sf.Sketch(4, 3001, 16, 13, 5, 4096, shared_dict=True)
    e = sf.Sketch(4, 3001, 16, 13, 5, 4096)
    bt = sf.Batch(2, dict_arena_bytes=need)
    torch.cuda.synchronize()
    bt.arena.fill_(0x11)
    bt.scratch[0] = 2
    torch.cuda.synchronize()
    assert bt.sync_status() == sf.SF_ERR_TIMEOUT
    assert int(torch.count_nonzero(bt.arena)) == 0
    bt.update([(c, ins, None)])
    e.insert(ins)
    assert bt.sync_status() == sf.SF_OK and e.sync_status() == sf.SF_OK
    assert torch.equal(c.fat, e.fat) and torch.equal(c.slim, e.slim)
    bt.close()
