"""Keys, operations and query answers in page-locked host memory: the kernels read and write
them over the host link themselves.  Results must be bit-identical to device-resident buffers
on every path (chunked, S = 1, batched, queries), and pageable host memory is refused before
anything is launched."""
import ctypes

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


def _pinned(t):
    return t.cpu().pin_memory()


@pytest.mark.parametrize("kb,S", [(4, 65536), (13, 4096), (4, 1), (13, 1)])
def test_pinned_keys_update_like_device_keys(sf, kb, S):
    import torch
    st, ids = wl.mixed_stream(60_000, 3_000, 1.1, 0.2, 4, seed=kb * 10 + S % 7)
    keys = st.keys if kb == 4 else torch.cat([st.keys, st.keys, st.keys, st.keys[:, :1]], 1).contiguous()
    qk = ids if kb == 4 else torch.cat([ids, ids, ids, ids[:, :1]], 1).contiguous()
    a = sf.Sketch(4, 1 << 12, 16, kb, 3, S)
    b = sf.Sketch(4, 1 << 12, 16, kb, 3, S)
    a.update(keys.cuda(), st.ops.cuda())
    b.update(_pinned(keys), _pinned(st.ops))
    a.sync()
    b.sync()
    assert torch.equal(a.fat, b.fat) and torch.equal(a.slim, b.slim)
    slim, hdr = b.export_slim()
    want = sf.query(slim, hdr, qk.cuda())
    got = sf.query(slim, hdr, _pinned(qk))          # answers land in pinned host memory
    torch.cuda.synchronize()
    assert got.device.type == "cpu" and got.is_pinned()
    assert torch.equal(want.cpu(), got)


def test_pinned_keys_in_a_batch(sf):
    import torch
    plan = wl.many_sketch_plan(8, seed=4, w_log2=(7.0, 10.0), n_log10=(3.0, 4.5))
    streams = [wl.mixed_stream(p["n"], p["distinct"], p["s"], 0.1, 4, seed=p["seed"])[0] for p in plan]
    chunks = [max(2, -(-p["n"] // 6)) for p in plan]
    dev_sk = [sf.Sketch(4, p["w"], 16, 4, p["seed"], S) for p, S in zip(plan, chunks)]
    host_sk = [sf.Sketch(4, p["w"], 16, 4, p["seed"], S) for p, S in zip(plan, chunks)]
    b1, b2 = sf.Batch(len(plan)), sf.Batch(len(plan))
    b1.update([(sk, s.keys.cuda(), s.ops.cuda()) for sk, s in zip(dev_sk, streams)])
    pinned = [(_pinned(s.keys), _pinned(s.ops)) for s in streams]
    b2.update([(sk, k, o) for sk, (k, o) in zip(host_sk, pinned)])
    assert b1.sync_status() == sf.SF_OK and b2.sync_status() == sf.SF_OK
    for x, y in zip(dev_sk, host_sk):
        assert torch.equal(x.fat, y.fat) and torch.equal(x.slim, y.slim)
    b1.close()
    b2.close()


def test_pageable_host_memory_is_refused_before_launch(sf):
    L = sf.load()
    g = sf.Sketch(2, 64, 4, 4, 1, 1024)
    keys = np.arange(100, dtype=np.uint32)          # ordinary (pageable) host memory
    assert L.sf_insert_batch(g.handle, keys.ctypes.data, 100) == sf.SF_ERR_INVALID
    out = np.zeros(100, dtype=np.uint32)
    slim, hdr = g.export_slim()
    v = sf.SlimView(slim.data_ptr(), hdr, 0, 0)
    assert L.sf_query_batch(ctypes.byref(v), keys.ctypes.data, 100, out.ctypes.data, None) == sf.SF_ERR_INVALID
    with pytest.raises(ValueError):
        import torch
        g.insert(torch.from_numpy(keys))             # the binding refuses it too
    assert g.sync_status() == sf.SF_OK               # nothing ran, nothing latched


@pytest.mark.parametrize("kb,S,with_ops", [(13, 4096, False), (4, 1000, True), (8, 65536, True), (4, 1, False)])
def test_pipelined_update_from_host_equals_one_call(sf, kb, S, with_ops):
    """sf_update_pipelined: host keys copied in chunk-aligned pieces through a small staging buffer
    (several pieces, both halves reused), overlapped with the updates, leave every counter equal to
    one sf_update_batch call over the whole stream; deletions through op_const as well."""
    import torch
    if kb == 13:
        ins, dels, _ = wl.flows_with_deletes(150_000, 20_000, 1.0, 0.1, seed=61)
        calls = [(ins, None, 1), (dels, None, -1)]
    else:
        st, _ = wl.mixed_stream(150_000, 20_000, 1.0, 0.2 if with_ops else 0.0, kb, seed=62)
        calls = [(st.keys, st.ops if with_ops else None, 1)]
    a = sf.Sketch(4, 2000, 16, kb, 5, S)
    b = sf.Sketch(4, 2000, 16, kb, 5, S)
    per = kb + (1 if with_ops else 0)
    staging = torch.empty(2 * (max(S, 7000) * per + 16) + 64, dtype=torch.uint8, device="cuda")
    for keys, ops, op_const in calls:
        kd = keys.cuda()
        if ops is not None:
            a.update(kd, ops.cuda())
        elif op_const > 0:
            a.insert(kd)
        else:
            a.delete(kd)
        b.update_pipelined(_pinned(keys), _pinned(ops) if ops is not None else None, op_const, staging=staging)
        a.sync()
        b.sync()
        assert torch.equal(a.fat, b.fat) and torch.equal(a.slim, b.slim)
    with pytest.raises(sf.SFError) as ei:
        b.update_pipelined(_pinned(calls[0][0]), None, 1, staging=torch.empty(16, dtype=torch.uint8, device="cuda"))
    assert ei.value.status == sf.SF_ERR_OOM


@pytest.mark.parametrize("kb,S,with_ops", [(13, 1000, True), (13, 999, False), (4, 1001, True), (8, 4096, True)])
def test_pipelined_staging_at_the_documented_minimum(sf, kb, S, with_ops):
    """Staging of exactly 2 * (chunk * (key_bytes + ops) + 32) bytes, 16-byte aligned, holds a piece
    of one chunk whatever the padding of its keys: here every piece is one chunk (both halves reused
    many times, a ragged last piece) and the counters equal one device-resident call.  Less than two
    chunks' bytes is SF_ERR_OOM; a staging buffer off a 16-byte boundary is SF_ERR_INVALID."""
    import torch
    st, _ = wl.mixed_stream(7 * S + 123, 3_000, 1.0, 0.2 if with_ops else 0.0, 4, seed=kb + S)
    keys = st.keys if kb == 4 else torch.cat([st.keys] * 4, 1)[:, :kb].contiguous()
    per = kb + (1 if with_ops else 0)
    a = sf.Sketch(4, 1500, 16, kb, 6, S)
    b = sf.Sketch(4, 1500, 16, kb, 6, S)
    ops = st.ops if with_ops else None
    if ops is not None:
        a.update(keys.cuda(), ops.cuda())
    else:
        a.insert(keys.cuda())
    staging = torch.empty(2 * (S * per + 32), dtype=torch.uint8, device="cuda")
    b.update_pipelined(_pinned(keys), _pinned(ops) if ops is not None else None, 1, staging=staging)
    a.sync()
    b.sync()
    assert torch.equal(a.fat, b.fat) and torch.equal(a.slim, b.slim)
    small = torch.empty(2 * S * per - 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(sf.SFError) as ei:
        b.update_pipelined(_pinned(keys), _pinned(ops) if ops is not None else None, 1, staging=small)
    assert ei.value.status == sf.SF_ERR_OOM
    off = torch.empty(2 * (S * per + 32) + 16, dtype=torch.uint8, device="cuda")[8:]
    with pytest.raises(sf.SFError) as ei:
        b.update_pipelined(_pinned(keys), _pinned(ops) if ops is not None else None, 1, staging=off)
    assert ei.value.status == sf.SF_ERR_INVALID
    assert b.sync_status() == sf.SF_OK


@pytest.mark.gpu
def test_pipeline_kept_across_calls_and_sketches(sf):
    """sf_update_pipeline: one pipeline (small staging: several pieces per call) serves calls of two
    sketches of different key widths and chunk sizes, on two streams, with no sync between calls;
    every counter equals the device-resident calls'.  A chunk larger than half the staging is
    SF_ERR_OOM; a misaligned staging buffer is refused."""
    import torch
    ins, dels, _ = wl.flows_with_deletes(120_000, 15_000, 1.0, 0.1, seed=71)
    st8, _ = wl.mixed_stream(150_000, 20_000, 1.2, 0.2, 8, seed=72)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    a1, b1 = sf.Sketch(4, 3001, 16, 13, 5, 4096), sf.Sketch(4, 3001, 16, 13, 5, 4096, stream=s1)
    a2, b2 = sf.Sketch(3, 2000, 8, 8, 9, 9000), sf.Sketch(3, 2000, 8, 8, 9, 9000, stream=s2)
    pipe = sf.Pipeline(staging_bytes=2 * (20_000 * 9 + 16))
    half = st8.keys.shape[0] // 2
    calls = [(a1, b1, ins, None, 1), (a2, b2, st8.keys[:half], st8.ops[:half], 1), (a1, b1, dels, None, -1),
             (a2, b2, st8.keys[half:], st8.ops[half:], 1)]
    for a, b, keys, ops, op_const in calls:
        kd = keys.contiguous().cuda()
        if ops is not None:
            a.update(kd, ops.contiguous().cuda())
        elif op_const > 0:
            a.insert(kd)
        else:
            a.delete(kd)
        b.update_through(pipe, _pinned(keys.contiguous()), _pinned(ops.contiguous()) if ops is not None else None,
                         op_const)
    for s in (a1, a2, b1, b2):
        s.sync()
    assert torch.equal(a1.fat, b1.fat) and torch.equal(a1.slim, b1.slim)
    assert torch.equal(a2.fat, b2.fat) and torch.equal(a2.slim, b2.slim)
    pipe.release_inputs()
    big = sf.Sketch(4, 2000, 16, 13, 5, 65536)
    with pytest.raises(sf.SFError) as ei:
        big.update_through(pipe, _pinned(ins[:70_000].contiguous()))
    assert ei.value.status == sf.SF_ERR_OOM
    pipe.close()
    L = sf.load()
    buf = torch.empty(4096, dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p()
    assert L.sf_pipeline_create(buf.data_ptr() + 8, 1024, 0, ctypes.byref(h)) == sf.SF_ERR_INVALID


def test_update_calls_stage_pinned_keys_through_the_idle_dictionary_half(sf):
    """Update calls on pinned host keys of sketches whose chunk rounds run the single-iteration
    kernel (chunk <= 65,536) stage them through the idle upper half of the sketch's dictionary
    region (pieces of whole chunks on a copy stream of the sketch's own).  Several staged calls
    (insertions, deletions, mixed operations; several pieces each and one short piece), device-key
    calls between them, and then a batch of two such sketches -- whose multi-iteration launch reads
    the whole region as its dictionary, so the staged bytes must have been zeroed -- all leave the
    counters equal to the same calls made with device keys."""
    import torch
    ins, dels, _ = wl.flows_with_deletes(1_400_000, 60_000, 1.0, 0.1, seed=95)
    st, _ = wl.mixed_stream(700_000, 30_000, 1.1, 0.2, 4, seed=96)
    keys13 = torch.cat([st.keys] * 4, 1)[:, :13].contiguous()
    a1, b1 = sf.Sketch(4, 20011, 16, 13, 7, 65536), sf.Sketch(4, 20011, 16, 13, 7, 65536)
    a2, b2 = sf.Sketch(4, 5003, 16, 13, 8, 4096), sf.Sketch(4, 5003, 16, 13, 8, 4096)
    calls = [
        (a1, b1, ins, None, 1),              # 22 chunks: several pieces of 9 chunks
        (a1, b1, keys13, st.ops, 0),         # mixed operations, staged with their ops
        (a2, b2, ins[:30_000], None, 1),     # one piece (9 chunks of 4,096 hold 36,864 updates)
        (a1, b1, dels, None, -1),
    ]
    held = []                                # host buffers stay alive until the sketches synced
    for a, b, keys, ops, op in calls:
        kd = keys.cuda()
        kh = _pinned(keys)
        oh = _pinned(ops) if ops is not None else None
        held += [kh, oh]
        if ops is not None:
            a.update(kd, ops.cuda())
            b.update(kh, oh)
        elif op > 0:
            a.insert(kd)
            b.insert(kh)
        else:
            a.delete(kd)
            b.delete(kh)
        b.insert(ins[:5_000].cuda())         # a device-key call between staged calls
        a.insert(ins[:5_000].cuda())
    for s in (a1, b1, a2, b2):
        assert s.sync_status() == sf.SF_OK
    assert torch.equal(a1.fat, b1.fat) and torch.equal(a1.slim, b1.slim)
    assert torch.equal(a2.fat, b2.fat) and torch.equal(a2.slim, b2.slim)
    # two chunks of 65,536 in one round: the multi-iteration kernel, over both whole regions
    more = ins[200_000:500_000].cuda()
    for x, y in ((a1, a2), (b1, b2)):
        bt = sf.Batch(2)
        bt.update([(x, more, None), (y, more[:100_000], None)])
        assert bt.sync_status() == sf.SF_OK
        bt.close()
    assert torch.equal(a1.fat, b1.fat) and torch.equal(a1.slim, b1.slim)
    assert torch.equal(a2.fat, b2.fat) and torch.equal(a2.slim, b2.slim)
    # and staged again after the batch
    kh = _pinned(ins[:300_000])
    a1.insert(ins[:300_000].cuda())
    b1.insert(kh)
    assert a1.sync_status() == sf.SF_OK and b1.sync_status() == sf.SF_OK
    assert torch.equal(a1.fat, b1.fat) and torch.equal(a1.slim, b1.slim)
