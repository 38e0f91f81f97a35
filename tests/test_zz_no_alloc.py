"""sf_update_batch_noalloc -- the update for callers that cannot allocate device memory.

It keeps its dictionary in the library's own fixed device array instead of a caller scratch
buffer.  These tests drive it through the C ABI and check, after each of two calls in a row,
that every Fat and Slim counter equals both what the regular entry point (sf_update_batch)
produces on the same stream and what the CPU oracle's chunked semantics give (integer counters:
equality), and that the call reports no device error.  The file is collected last on purpose."""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def test_noalloc_update_matches_regular_update_twice(sf):
    import torch
    d, w, z, kb, seed, S = 4, 1 << 12, 16, 13, 7, 4096
    flows_a = wl.flows_with_deletes(40_000, 5_000, 1.0, 0.1, seed=43)
    calls = [(flows_a[0], None), (flows_a[1], "del")]
    regular = sf.Sketch(d, w, z, kb, seed, S)
    params = sf.make_params(d, w, z, kb, seed, S)
    o = oracle.Sketch(d, w, z, kb, seed)
    fat = torch.zeros(d * w * z, dtype=torch.int32, device="cuda")
    slim = torch.zeros(d * w, dtype=torch.int32, device="cuda")
    err = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for keys, kind in calls:
        kd = keys.cuda()
        ops = torch.full((kd.shape[0],), -1 if kind == "del" else 1, dtype=torch.int8, device="cuda")
        regular.update(kd, ops)
        sf.update_batch_noalloc(params, fat, slim, kd, ops, err)
        o.update(keys.numpy(), ops.cpu().numpy(), S=S)
        regular.sync()
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        assert torch.equal(fat, regular.fat), "Fat counters differ from sf_update_batch"
        assert torch.equal(slim, regular.slim), "Slim counters differ from sf_update_batch"
        assert np.array_equal(_u32(fat).reshape(d, w, z), o.B), "Fat counters differ from the oracle"
        assert np.array_equal(_u32(slim).reshape(d, w), o.A), "Slim counters differ from the oracle"


def test_noalloc_u32_mixed_stream_and_limits(sf):
    import torch
    d, w, z, kb, seed = 3, 997, 8, 4, 11
    st, _ = wl.mixed_stream(50_000, 4_000, 1.1, 0.25, 4, seed=44)
    half = 20_001
    err = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for S in (2, 1000, 16384):
        regular = sf.Sketch(d, w, z, kb, seed, S)
        params = sf.make_params(d, w, z, kb, seed, S)
        o = oracle.Sketch(d, w, z, kb, seed)
        fat = torch.zeros(d * w * z, dtype=torch.int32, device="cuda")
        slim = torch.zeros(d * w, dtype=torch.int32, device="cuda")
        for lo, hi in ((0, half), (half, st.keys.shape[0])):
            k = st.keys[lo:hi].cuda()
            op = st.ops[lo:hi].cuda()
            regular.update(k, op)
            sf.update_batch_noalloc(params, fat, slim, k, op, err)
            o.update(st.keys[lo:hi].numpy(), st.ops[lo:hi].numpy(), S=S)
            regular.sync()
            torch.cuda.synchronize()
            assert int(err.item()) == 0, (S, lo)
            assert torch.equal(fat, regular.fat) and torch.equal(slim, regular.slim), (S, lo)
            assert np.array_equal(_u32(fat).reshape(d, w, z), o.B), (S, lo)
            assert np.array_equal(_u32(slim).reshape(d, w), o.A), (S, lo)
    too_big = sf.make_params(d, w, z, kb, seed, 16385)
    with pytest.raises(sf.SFError) as ei:
        sf.update_batch_noalloc(too_big, fat, slim, st.keys[:10].cuda())
    assert ei.value.status == sf.SF_ERR_INVALID
    explicit = sf.make_params(d, w, z, kb, seed, 64, sf.SF_FLAG_EXPLICIT_INDEX)
    with pytest.raises(sf.SFError) as ei:
        sf.update_batch_noalloc(explicit, fat, slim, st.keys[:10].cuda())
    assert ei.value.status == sf.SF_ERR_INVALID
