"""GPU parity: every Fat counter, every Slim counter and every query answer of the CUDA path,
bit-exact against the CPU oracle on the same seeded inputs (integer work: no tolerance)."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _np_u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


def _run_both(sf, d, w, z, kb, seed, S, calls, rule="sff"):
    """calls: list of (keys uint8 (n,kb) cpu tensor, ops int8 cpu tensor or None=insert or 'del')."""
    import torch
    g = sf.Sketch(d, w, z, kb, seed, S, delete_rule=rule)
    o = oracle.Sketch(d, w, z, kb, seed, delete_rule=rule)
    for keys, ops in calls:
        kd = keys.cuda()
        if isinstance(ops, str) and ops == "del":
            g.delete(kd)
            o.update(keys.numpy(), -np.ones(len(keys), np.int8), S=S)
        elif ops is None:
            g.insert(kd)
            o.update(keys.numpy(), np.ones(len(keys), np.int8), S=S)
        else:
            g.update(kd, ops.cuda())
            o.update(keys.numpy(), ops.numpy(), S=S)
    g.sync()
    return g, o


def _assert_same(g, o):
    A = _np_u32(g.slim_view())
    B = _np_u32(g.fat_view())
    assert np.array_equal(B, o.B), f"Fat differs at {np.argwhere(B != o.B)[:5].tolist()}"
    assert np.array_equal(A, o.A), f"Slim differs at {np.argwhere(A != o.A)[:5].tolist()}"


def _queries_match(sf, g, o, qkeys):
    slim, hdr = g.export_slim()
    got = _np_u32(sf.query(slim, hdr, qkeys.cuda()))
    want = o.query(qkeys.numpy())
    assert np.array_equal(got, want)


def test_worked_example_sec32_on_gpu(sf):
    import torch
    gold = json.load(open(os.path.join(GOLD, "worked_example_fig3.json")))
    for S in (1, 2):
        for fchoice in gold["fat_slot_choices"]:
            table = np.zeros((2, 2, 2), np.uint32)
            for k, name in enumerate(("e1", "e2")):
                table[k, :, 0] = gold["keys"][name]["h"]
                table[k, :, 1] = fchoice[k]
            g = sf.Sketch(2, 2, 2, 4, 0, S, explicit_index=True)
            g.set_index_table(torch.from_numpy(table.view(np.int32)))
            ids = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
            g.insert(ids)
            g.sync()
            after_ins = _np_u32(g.slim_view()).tolist()
            g.delete(ids[:1].clone())
            g.sync()
            after_del = _np_u32(g.slim_view()).tolist()
            slim, hdr = g.export_slim()
            q = _np_u32(sf.query(slim, hdr, ids, index_table=g._index_table)).tolist()
            if S == 1:
                assert after_ins == gold["after_inserts_printed_by_paper"]["A"]
            assert after_del == gold["after_delete_e1_by_SF_F_rule"]["A"]
            assert q == [gold["after_delete_e1_by_SF_F_rule"]["query"]["e1"],
                         gold["after_delete_e1_by_SF_F_rule"]["query"]["e2"]]


@pytest.mark.parametrize("S", [1, 2, 7, 64, 1000, 4096, 65536])
def test_mixed_stream_u32(sf, S):
    st, ids = wl.mixed_stream(20_000, 3_000, 1.1, 0.3, 4, seed=11 + S)
    g, o = _run_both(sf, 4, 97, 16, 4, 5, S, [(st.keys, st.ops)])
    _assert_same(g, o)
    _queries_match(sf, g, o, ids)


@pytest.mark.parametrize("del_frac", [0.0, 0.02])
@pytest.mark.parametrize("d,w,z", [(4, 97, 16), (3, 1 << 16, 8)])
def test_one_at_a_time_windows(sf, del_frac, d, w, z):
    """S = 1 on streams whose windows mostly hold no deletion (the precomputed-Fat path), with
    deletion windows in between (the in-step path) and hot keys (several lanes on one counter).
    w = 2^16 puts the Slim (768 KiB) beyond shared memory, so the steps run on global memory."""
    st, ids = wl.mixed_stream(40_000, 1_500, 1.2, del_frac, 4, seed=int(del_frac * 100) + w)
    g, o = _run_both(sf, d, w, z, 4, 9, 1, [(st.keys, st.ops)])
    _assert_same(g, o)
    _queries_match(sf, g, o, ids)


@pytest.mark.parametrize("d,w,z,kb,s_,n", [
    (4, 4096, 16, 4, 1.0, 100_000),      # the C1 shape
    (1, 1024, 16, 4, 1.5, 50_000),       # one row, hot keys: long runs
    (8, 2048, 7, 13, 1.1, 60_000),       # eight rows, 13-byte keys, odd bucket size
    (3, 1 << 14, 16, 8, 0.8, 300_001),   # several pieces of the graph path, a ragged last one
])
def test_one_at_a_time_insertions_graph_path(sf, d, w, z, kb, s_, n):
    """S = 1 insertion-only calls on sketches of width >= 1024 take the dependency-graph path:
    every counter and query equals the oracle's literal one-at-a-time rule, over two calls."""
    import torch
    st, ids = wl.mixed_stream(n, 5_000, s_, 0.0, 4, seed=d * 1000 + w % 997 + n % 13)
    keys = st.keys if kb == 4 else torch.cat([st.keys] * 4, 1)[:, :kb].contiguous()
    qk = ids if kb == 4 else torch.cat([ids] * 4, 1)[:, :kb].contiguous()
    h = n // 3
    g, o = _run_both(sf, d, w, z, kb, 21, 1, [(keys[:h], None), (keys[h:], None)])
    _assert_same(g, o)
    _queries_match(sf, g, o, qk)


@pytest.mark.parametrize("d,z", [(2, 16), (5, 3), (6, 16), (7, 5)])
def test_one_at_a_time_graph_path_every_row_count(sf, d, z):
    """The graph walk is compiled for each d: the row counts the shapes above do not reach, with
    Zipf-hot keys (long runs) over two calls."""
    st, ids = wl.mixed_stream(30_000, 3_000, 1.2, 0.0, 4, seed=600 + d)
    g, o = _run_both(sf, d, 1024 + 64 * d, z, 4, 11, 1, [(st.keys[:10_001], None), (st.keys[10_001:], None)])
    _assert_same(g, o)
    _queries_match(sf, g, o, ids)


def test_one_at_a_time_graph_path_wide_frontier(sf):
    """Uniform keys over many more ids than one piece holds: most updates start with no
    predecessor, so the first frontiers overflow the walk's shared-memory queues into the global
    ones; two pieces."""
    st, ids = wl.mixed_stream(200_000, 1_000_000, 0.0, 0.0, 8, seed=4242)
    g, o = _run_both(sf, 4, 1 << 17, 16, 8, 3, 1, [(st.keys, None)])
    _assert_same(g, o)
    _queries_match(sf, g, o, ids[:50_000])


def test_one_at_a_time_graph_path_pinned_keys_and_explicit_ids(sf):
    import torch
    st, ids = wl.mixed_stream(40_000, 2_000, 1.2, 0.0, 4, seed=77)
    a = sf.Sketch(4, 2048, 16, 4, 5, 1)
    b = sf.Sketch(4, 2048, 16, 4, 5, 1)
    a.insert(st.keys.cuda())
    b.insert(st.keys.cpu().pin_memory())
    a.sync()
    b.sync()
    assert torch.equal(a.fat, b.fat) and torch.equal(a.slim, b.slim)
    # explicit-index mode: key ids into a table of (h_i, f_i)
    gen = np.random.default_rng(3)
    table = np.stack([gen.integers(0, 2048, (500, 4)), gen.integers(0, 16, (500, 4))], axis=2).astype(np.uint32)
    idx = gen.integers(0, 500, 30_000).astype(np.uint32)
    g = sf.Sketch(4, 2048, 16, 4, 0, 1, explicit_index=True)
    g.set_index_table(torch.from_numpy(table.view(np.int32)).cuda())
    g.insert(torch.from_numpy(idx.view(np.int32)).cuda())
    g.sync()
    o = oracle.Sketch(4, 2048, 16, 4, 0)
    hh, ff, ident = oracle.explicit_indices(table, idx)
    o.seq_apply(hh, ff, np.ones(len(idx), np.int8))
    _assert_same(g, o)


@pytest.mark.parametrize("w,S", [(2048, 1), (500, 1), (2048, 4096)])
def test_explicit_ids_out_of_range_are_skipped_and_reported(sf, w, S):
    """Ids beyond the index table are reported (SF_ERR_INVALID at the next sync) and change no
    counter: the sketch equals the oracle's with those updates' operations set to 0 (the graph
    path, the one-warp window path and the chunked path)."""
    import torch
    gen = np.random.default_rng(17 + w + S)
    n_keys = 300
    table = np.stack([gen.integers(0, w, (n_keys, 4)), gen.integers(0, 16, (n_keys, 4))], axis=2).astype(np.uint32)
    ids = gen.integers(0, n_keys + 25, 20_000).astype(np.uint32)
    valid = ids < n_keys
    assert 0 < int((~valid).sum()) < len(ids)
    g = sf.Sketch(4, w, 16, 4, 0, S, explicit_index=True)
    g.set_index_table(torch.from_numpy(table.view(np.int32)).cuda())
    g.insert(torch.from_numpy(ids.view(np.int32)).cuda())
    assert g.sync_status() == sf.SF_ERR_INVALID
    o = oracle.Sketch(4, w, 16, 4, 0)
    hh, ff, ident = oracle.explicit_indices(table, np.where(valid, ids, 0).astype(np.uint32))
    ops = valid.astype(np.int8)
    if S == 1:
        o.seq_apply(hh, ff, ops)
    else:
        o.chunk_apply(hh, ff, ops, S, ids.view(np.uint8).reshape(-1, 4))
    _assert_same(g, o)


@pytest.mark.parametrize("n", [1, 31, 32, 33, 64, 65, 97])
def test_one_at_a_time_short_streams(sf, n):
    """S = 1 on lengths around the 32-update window and the two-window key prefetch."""
    st, ids = wl.mixed_stream(n, 7, 1.5, 0.0, 4, seed=n)
    g, o = _run_both(sf, 4, 5, 3, 4, 1, 1, [(st.keys, st.ops), (st.keys[: n // 2 + 1], None)])
    _assert_same(g, o)
    _queries_match(sf, g, o, ids)


@pytest.mark.parametrize("S", [1, 7, 4096, 65536])
@pytest.mark.parametrize("d,w,z", [(4, 97, 16), (3, 50, 7)])
def test_sf4_delete_rule(sf, S, d, w, z):
    """The SF_4 deletion (Sec. 3.4, clamp to the bucket sum) on turnstile streams; z = 7 takes
    the scalar bucket read, z = 16 the vector one."""
    st, ids = wl.mixed_stream(30_000, 2_000, 1.1, 0.3, 4, seed=900 + S + z)
    g, o = _run_both(sf, d, w, z, 4, 5, S, [(st.keys, st.ops)], rule="sf4")
    _assert_same(g, o)
    _queries_match(sf, g, o, ids)
    # Over several chunks the two rules give different sketches (the ablation compares two
    # different things).  Within a single chunk they cannot differ: every raise target is at
    # most the bucket maximum, so neither clamp binds.
    if S < st.keys.shape[0] // 2:
        f, _ = _run_both(sf, d, w, z, 4, 5, S, [(st.keys, st.ops)], rule="sff")
        assert not np.array_equal(_np_u32(f.slim_view()), _np_u32(g.slim_view()))


@pytest.mark.parametrize("kb", [1, 3, 8, 13, 15])
def test_key_widths(sf, kb):
    import torch
    gen = torch.Generator().manual_seed(kb)
    pool = torch.randint(0, 256, (500, kb), dtype=torch.uint8, generator=gen)
    pool = torch.unique(pool, dim=0)
    ranks = wl.sample_ranks(30_000, pool.shape[0], 1.2, gen)
    keys = pool[ranks].contiguous()
    ops = torch.where(torch.rand(30_000, generator=gen) < 0.15, -1, 1).to(torch.int8)
    # make the stream strict-turnstile: a delete only if that key has a live insert
    live = {}
    ok = []
    for t in range(len(keys)):
        kk = bytes(keys[t].tolist())
        if ops[t] < 0 and live.get(kk, 0) == 0:
            ops[t] = 1
        live[kk] = live.get(kk, 0) + int(ops[t])
    for S in (1, 333, 8192):
        g, o = _run_both(sf, 3, 50, 8, kb, 77, S, [(keys, ops)])
        _assert_same(g, o)
        _queries_match(sf, g, o, pool)


@pytest.mark.parametrize("kb", [1, 2, 3, 5, 6, 7, 9, 11, 12, 13, 14, 15])
def test_queries_with_unaligned_and_ragged_keys(sf, kb):
    """Point queries (Sec. 3.1) on keys of widths other than 4 and 8 bytes, which the query kernels
    read as the aligned 8-byte words covering each key (byte loads where those words would leave
    the buffer): key buffers starting at every offset 0..15 bytes past a 16-byte boundary, lengths
    that leave a ragged last warp (1, 31, 33, 100,003 keys), answers equal the oracle's."""
    import torch
    gen = torch.Generator().manual_seed(200 + kb)
    pool = torch.unique(torch.randint(0, 256, (4000, kb), dtype=torch.uint8, generator=gen), dim=0)
    keys = pool[wl.sample_ranks(60_000, pool.shape[0], 1.0, gen)].contiguous()
    g, o = _run_both(sf, 4, 3001, 16, kb, 5, 4096, [(keys, None)])
    slim, hdr = g.export_slim()
    q = pool[torch.randint(0, pool.shape[0], (100_003 + 16,), generator=gen)].contiguous()
    flat = q.view(-1).cuda()
    for off in range(16):
        for n in (1, 31, 33, 100_003):
            dev = flat[off: off + n * kb]          # starts off bytes past the allocation's alignment
            want = o.query(q.view(-1)[off: off + n * kb].view(n, kb).numpy())
            got = _np_u32(sf.query(slim, hdr, dev.view(n, kb)))
            assert np.array_equal(got, want), (off, n)


@pytest.mark.parametrize("d,w,z", [(1, 1, 1), (2, 5, 3), (5, 300, 7), (6, 777, 9), (7, 1500, 16), (8, 4096, 16),
                                   (4, 1 << 12, 64)])
def test_shapes(sf, d, w, z):
    st, ids = wl.mixed_stream(12_345, 2_000, 0.9, 0.25, 4, seed=d * 100 + z)
    for S in (1, 3, 4096):
        g, o = _run_both(sf, d, w, z, 4, 3, S, [(st.keys, st.ops)])
        _assert_same(g, o)
        _queries_match(sf, g, o, ids)


def test_insert_then_delete_calls_restart_chunks(sf):
    ins, dels, flows = wl.flows_with_deletes(200_000, 20_000, 1.0, 0.1, seed=3)
    for S in (65536, 50_000):
        g, o = _run_both(sf, 4, 1 << 12, 16, 13, 2, S, [(ins[:123_457], None), (ins[123_457:], None), (dels, "del")])
        _assert_same(g, o)
        _queries_match(sf, g, o, flows)


def test_empty_and_tiny_batches(sf):
    import torch
    g = sf.Sketch(4, 64, 16, 4, 1, 64)
    g.insert(torch.empty(0, dtype=torch.int32, device="cuda"))
    g.sync()
    assert int(g.slim.abs().sum()) == 0 and int(g.fat.abs().sum()) == 0
    o = oracle.Sketch(4, 64, 16, 4, 1)
    k = torch.tensor([5], dtype=torch.int32)
    g.insert(k.cuda())
    g.sync()
    o.update(k.numpy().view(np.uint8).reshape(-1, 4), np.ones(1, np.int8), S=64)
    _assert_same(g, o)
    slim, hdr = g.export_slim()
    assert sf.query(slim, hdr, torch.empty(0, dtype=torch.int32, device="cuda")).numel() == 0


def test_theorem_error_free_fat_on_gpu(sf):
    """Sec. 3.5 Theorem 1 through the GPU path (explicit indices, insertions only)."""
    import torch
    rng = np.random.default_rng(17)
    n_keys, d, w, z = 200, 3, 32, 16
    table = np.zeros((n_keys, d, 2), np.uint32)
    for i in range(d):
        used = np.zeros(w, np.int64)
        for k in range(n_keys):
            j = int(rng.integers(w))
            while used[j] >= z:
                j = int(rng.integers(w))
            table[k, i] = (j, used[j])
            used[j] += 1
    ids = ((rng.zipf(1.2, 50_000) - 1) % n_keys).astype(np.uint32)
    freq = np.bincount(ids, minlength=n_keys)
    want = np.zeros((d, w), np.int64)
    for k in range(n_keys):
        for i in range(d):
            want[i, table[k, i, 0]] = max(want[i, table[k, i, 0]], freq[k])
    for S in (1, 5, 4096):
        g = sf.Sketch(d, w, z, 4, 0, S, explicit_index=True)
        g.set_index_table(torch.from_numpy(table.view(np.int32)))
        g.insert(torch.from_numpy(ids.view(np.int32)).cuda())
        g.sync()
        assert np.array_equal(_np_u32(g.slim_view()).astype(np.int64), want)


def test_underflow_is_reported(sf):
    import torch
    for S in (1, 16):
        g = sf.Sketch(2, 16, 4, 4, 9, S)
        g.delete(torch.tensor([42], dtype=torch.int32, device="cuda"))
        assert g.sync_status() == sf.SF_ERR_UNDERFLOW
        assert g.sync_status() == sf.SF_OK  # cleared after being reported


def test_bad_key_id_in_explicit_mode_is_reported(sf):
    import torch
    for S in (1, 8):
        g = sf.Sketch(2, 4, 4, 4, 0, S, explicit_index=True)
        g.set_index_table(torch.zeros((3, 2, 2), dtype=torch.int32))
        g.insert(torch.tensor([0, 7], dtype=torch.int32, device="cuda"))
        assert g.sync_status() == sf.SF_ERR_INVALID


def test_flows_zipf_sweep_mid_size(sf):
    """Shape of the 5-tuple workload (13-byte keys, Zipf sweep, inserts then 10 % deletes,
    chunk 65,536) at 1/64 of its stream length and Slim width."""
    for s in wl.ZIPF_SWEEP:
        ins, dels, flows = wl.flows_with_deletes(500_000, 16_384, s, 0.1, seed=int(s * 10) + 1)
        g, o = _run_both(sf, 4, 1 << 12, 16, 13, 2, 65536, [(ins, None), (dels, "del")])
        _assert_same(g, o)
        _queries_match(sf, g, o, flows)


def test_query_pipeline_splits_like_the_paper_and_matches(sf):
    """Sec. 4.2.2 multi-stream pipeline: parts of nearly equal size over n streams (the first
    b % n take one more); answers equal one sf_query_batch over the whole batch."""
    import torch
    st, ids = wl.mixed_stream(50_000, 8_000, 1.0, 0.2, 4, seed=91)
    g = sf.Sketch(4, 2048, 16, 4, 3, 1000)
    g.update(st.keys.cuda(), st.ops.cuda())
    slim, hdr = g.export_slim()
    g.sync()
    keys = torch.cat([ids, ids[:1234]]).contiguous()
    want = _np_u32(sf.query(slim, hdr, keys.cuda()))
    for n_streams in (1, 3, 7, 16):
        streams = [torch.cuda.Stream() for _ in range(n_streams)]
        kh = keys.pin_memory()
        oh = torch.zeros(keys.shape[0], dtype=torch.int32).pin_memory()
        kd = torch.empty_like(keys, device="cuda")
        od = torch.empty(keys.shape[0], dtype=torch.int32, device="cuda")
        sf.query_pipelined(slim, hdr, kh, oh, kd, od, streams)
        for s_ in streams:
            s_.synchronize()
        assert np.array_equal(oh.numpy().view(np.uint32), want), n_streams


@pytest.mark.parametrize("S", [1, 64, 4096])
def test_correct_rate_bound_eq_cr_on_gpu(sf, S):
    """Sec. 3.5, Eq. (cr), through the CUDA path: v items of frequencies 1..v over an error-free
    Fat (explicit indices, no two items on one Fat counter), d = 3, w = 64.  The share of items the
    GPU's Slim answers exactly is at least (1/v) sum_l [1 - (1 - (1 - 1/w)^(v-l))^d] (averaged over
    trials, 0.02 slack); every counter also equals the oracle's (SEQ for S = 1, chunked otherwise;
    with an error-free Fat both give each Slim counter its maximum true frequency, Sec. 3.5)."""
    import torch
    from tests.test_oracle_pins import _collision_free_fat_table
    v, d, w, z = 120, 3, 64, 64
    bound = np.mean([1 - (1 - (1 - 1 / w) ** (v - l)) ** d for l in range(1, v + 1)])
    rates = []
    for trial in range(12):
        rng = np.random.default_rng(1000 + trial)
        table = _collision_free_fat_table(rng, v, d, w, z)
        ids = np.repeat(np.arange(v, dtype=np.uint32), np.arange(1, v + 1))
        rng.shuffle(ids)
        g = sf.Sketch(d, w, z, 4, 0, S, explicit_index=True)
        g.set_index_table(torch.from_numpy(table.astype(np.int32)))
        g.insert(torch.from_numpy(ids.astype(np.int32)).cuda())
        slim, hdr = g.export_slim()
        q = _np_u32(sf.query(slim, hdr, torch.arange(v, dtype=torch.int32, device="cuda"),
                             index_table=g._index_table))
        g.sync()
        o = oracle.Sketch(d, w, z)
        h, f, ident = oracle.explicit_indices(table, ids)
        if S == 1:
            o.seq_apply(h, f, np.ones(len(ids), np.int8))
        else:
            o.chunk_apply(h, f, np.ones(len(ids), np.int8), S, ident)
        assert np.array_equal(_np_u32(g.slim_view()), o.A) and np.array_equal(_np_u32(g.fat_view()), o.B)
        rates.append(float(np.mean(q == np.arange(1, v + 1))))
    assert np.mean(rates) >= bound - 0.02


@pytest.mark.parametrize("S", [1, 4096, 65536])
def test_reset_equals_a_fresh_sketch(sf, S):
    """sf_reset (Sec. 3.1 initialisation on the same buffers) zeroes Fat, Slim and control words;
    the dictionary left zeroed by the previous calls is reused: a reset sketch fed a stream ends
    with exactly the counters of a fresh sketch fed the same stream (and of the oracle)."""
    import torch
    ins, dels, flows = wl.flows_with_deletes(120_000, 9_000, 1.1, 0.1, seed=71)
    g = sf.Sketch(4, 3000, 16, 13, 4, S)
    g.insert(ins.cuda())
    g.delete(dels.cuda())
    g.sync()
    g.reset()
    g.insert(ins[:70_000].cuda())
    g.sync()
    o = oracle.Sketch(4, 3000, 16, 13, 4)
    o.update(ins[:70_000].numpy(), np.ones(70_000, np.int8), S=S)
    _assert_same(g, o)


@pytest.mark.parametrize("S", [65_536, 65_537])
def test_both_update_kernels_at_the_chunk_size_boundary(sf, S):
    """S = 65,536 is the largest chunk of the single-iteration kernel (16-bit claim positions and
    counts; the hot key of a Zipf-3 stream fills most of a chunk, so its counts approach that limit),
    S = 65,537 runs the multi-iteration kernel: both equal the oracle, with ragged last chunks and a
    mixed stream."""
    ins, dels, flows = wl.flows_with_deletes(400_003, 40_000, 3.0, 0.1, seed=81)
    g, o = _run_both(sf, 4, 1 << 12, 16, 13, 9, S, [(ins, None), (dels, "del")])
    _assert_same(g, o)
    _queries_match(sf, g, o, flows)
    st, ids = wl.mixed_stream(300_001, 30_000, 1.2, 0.2, 8, seed=82)
    g, o = _run_both(sf, 4, 5000, 16, 8, 9, S, [(st.keys, st.ops)])
    _assert_same(g, o)


@pytest.mark.parametrize("S", [65_536, 1 << 20])
def test_maximum_parameters(sf, S):
    """Every parameter at its limit at once: d = SF_MAX_D (8) rows, buckets of SF_MAX_Z (64)
    counters, SF_MAX_KEY_BYTES (15)-byte keys, and chunks of 65,536 (the single-iteration kernel's
    largest) or SF_MAX_CHUNK (2^20, multi-iteration) updates, over two whole chunks and a ragged
    tail of a strict-turnstile stream: counters and queries equal the oracle's."""
    import torch
    n = 2 * S + 12_345
    st, ids = wl.mixed_stream(n, 50_000, 1.0, 0.2, 8, seed=S % 997)
    keys = torch.cat([st.keys, st.keys], 1)[:, :15].contiguous()
    qk = torch.cat([ids, ids], 1)[:, :15].contiguous()
    g, o = _run_both(sf, 8, 3001, 64, 15, 11, S, [(keys, st.ops)])
    _assert_same(g, o)
    _queries_match(sf, g, o, qk)
