"""Batched many-sketch update (one persistent cooperative launch, CUDA graph replay): every
sketch's Fat and Slim equal those of one sf_update_batch call per sketch (bit for bit), and
sampled sketches equal the CPU oracle's chunked semantics with the same chunk size."""
import numpy as np
import pytest

import oracle
import workloads as wl
from paper_1701_04148_gb300 import shard

pytestmark = pytest.mark.gpu


def _plan(n_sketches, seed, w_log2=(6.0, 11.0), n_log10=(2.0, 4.7)):
    return wl.many_sketch_plan(n_sketches, seed, w_log2=w_log2, n_log10=n_log10)


def _streams(plan, device="cuda"):
    out = []
    for p in plan:
        st, ids = wl.mixed_stream(p["n"], p["distinct"], p["s"], 0.1, 4, seed=p["seed"], device=device)
        out.append((st, ids))
    return out


def _chunk_for(p, rounds):
    return max(2, -(-p["n"] // rounds))


@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_per_sketch_calls(sf, graph):
    import torch
    plan = _plan(37, seed=5)
    streams = _streams(plan)
    for rounds in (3, 40):
        batch_sk = [sf.Sketch(4, p["w"], 16, 4, p["seed"], _chunk_for(p, rounds)) for p in plan]
        plain_sk = [sf.Sketch(4, p["w"], 16, 4, p["seed"], _chunk_for(p, rounds)) for p in plan]
        b = sf.Batch(len(plan), graph=graph)
        halves = []
        for (st, _) in streams:
            h = st.keys.shape[0] // 2
            halves.append(((st.keys[:h], st.ops[:h]), (st.keys[h:], st.ops[h:])))
        for part in (0, 1):  # two calls in a row (graph replay when the shape repeats)
            b.update([(sk, halves[i][part][0], halves[i][part][1]) for i, sk in enumerate(batch_sk)])
            for i, sk in enumerate(plain_sk):
                sk.update(halves[i][part][0], halves[i][part][1])
        b.sync()
        for sk in plain_sk:
            sk.sync()
        for i in range(len(plan)):
            assert torch.equal(batch_sk[i].fat, plain_sk[i].fat), (rounds, i)
            assert torch.equal(batch_sk[i].slim, plain_sk[i].slim), (rounds, i)
        info = b.info()
        if graph:
            assert info["graph_captures"] >= 1 and info["graph_launches"] == 2
        b.close()


def test_batch_matches_oracle_on_sampled_sketches(sf):
    import torch
    plan = _plan(24, seed=9, w_log2=(7.0, 12.0), n_log10=(3.0, 5.0))
    streams = _streams(plan)
    sks = [sf.Sketch(4, p["w"], 16, 4, p["seed"], _chunk_for(p, 17)) for p in plan]
    b = sf.Batch(len(plan))
    b.update([(sk, st.keys, st.ops) for sk, (st, _) in zip(sks, streams)])
    b.sync()
    for i in (0, 5, 11, 23):
        p = plan[i]
        st, ids = streams[i]
        o = oracle.Sketch(4, p["w"], 16, 4, p["seed"])
        o.update(st.keys.cpu().numpy(), st.ops.cpu().numpy(), S=_chunk_for(p, 17))
        assert np.array_equal(sks[i].fat.cpu().numpy().view(np.uint32).reshape(o.B.shape), o.B)
        assert np.array_equal(sks[i].slim.cpu().numpy().view(np.uint32).reshape(o.A.shape), o.A)


@pytest.mark.parametrize("world,rank", [(2, 1), (3, 0)])
def test_one_ranks_share_of_a_sharded_batch(sf, world, rank):
    """The sharded many-sketch batch: one rank's share (shard.owned) of a batch of independent
    sketches, updated by one batched launch on this GPU, equals one sf_update_batch call per
    sketch, and sampled sketches of the share equal the oracle's chunked semantics."""
    import torch
    plan = _plan(30, seed=31, w_log2=(7.0, 11.0), n_log10=(2.5, 4.5))
    mine = shard.owned([p["n"] for p in plan], world, rank)
    assert 0 < len(mine) < len(plan)
    share = [plan[i] for i in mine]
    streams = _streams(share)
    chunks = [_chunk_for(p, 9) for p in share]
    bsk = [sf.Sketch(4, p["w"], 16, 4, p["seed"], c) for p, c in zip(share, chunks)]
    psk = [sf.Sketch(4, p["w"], 16, 4, p["seed"], c) for p, c in zip(share, chunks)]
    b = sf.Batch(len(share))
    b.update([(sk, st.keys, st.ops) for sk, (st, _) in zip(bsk, streams)])
    for sk, (st, _) in zip(psk, streams):
        sk.update(st.keys, st.ops)
    assert b.sync() == sf.SF_OK
    for sk in psk:
        sk.sync()
    for i in range(len(share)):
        assert torch.equal(bsk[i].fat, psk[i].fat) and torch.equal(bsk[i].slim, psk[i].slim), i
    for i in sorted({0, len(share) // 2, len(share) - 1}):
        p, (st, _) = share[i], streams[i]
        o = oracle.Sketch(4, p["w"], 16, 4, p["seed"])
        o.update(st.keys.cpu().numpy(), st.ops.cpu().numpy(), S=chunks[i])
        assert np.array_equal(bsk[i].fat.cpu().numpy().view(np.uint32).reshape(o.B.shape), o.B), mine[i]
        assert np.array_equal(bsk[i].slim.cpu().numpy().view(np.uint32).reshape(o.A.shape), o.A), mine[i]


@pytest.mark.parametrize("threads", [128, 256, 512])
def test_launch_shapes_give_the_same_sketches(sf, threads):
    """Every block shape of sf_batch_set_block_threads (512 / threads blocks per SM) leaves each
    sketch equal to one sf_update_batch call per sketch: rounds of a few thousand slots (one update
    per worker lane: the single-iteration kernel) and rounds of several hundred thousand (the
    multi-iteration kernel)."""
    import torch
    plan = _plan(20, seed=41, w_log2=(8.0, 12.0), n_log10=(3.0, 5.3))
    streams = _streams(plan)
    for rounds in (40, 2):
        chunks = [_chunk_for(p, rounds) for p in plan]
        bsk = [sf.Sketch(4, p["w"], 16, 4, p["seed"], c) for p, c in zip(plan, chunks)]
        psk = [sf.Sketch(4, p["w"], 16, 4, p["seed"], c) for p, c in zip(plan, chunks)]
        b = sf.Batch(len(plan), block_threads=threads, group_bytes=0)
        b.update([(sk, st.keys, st.ops) for sk, (st, _) in zip(bsk, streams)])
        for sk, (st, _) in zip(psk, streams):
            sk.update(st.keys, st.ops)
        assert b.sync() == sf.SF_OK
        for sk in psk:
            sk.sync()
        for i in range(len(plan)):
            assert torch.equal(bsk[i].fat, psk[i].fat) and torch.equal(bsk[i].slim, psk[i].slim), (threads, rounds, i)
        b.close()
    with pytest.raises(sf.SFError):
        sf.Batch(4, block_threads=384)


def test_batch_rounds_at_the_single_iteration_boundary(sf):
    """A batch whose rounds hold exactly one slot per worker lane of the grid (152 x 15 warps x 32 =
    72,960 slots on a 152-SM GB300: the single-iteration kernel) and one warp of slots more (the
    multi-iteration kernel): every sketch equals one sf_update_batch call and sampled sketches the
    oracle."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    lanes = sms * (512 - 32)
    for extra in (0, 32):
        # ten sketches whose chunk sizes (multiples of 32) sum to lanes + extra
        base = (lanes + extra) // 10 // 32 * 32
        chunks = [base] * 9 + [lanes + extra - 9 * base]
        plan = _plan(10, seed=51 + extra, w_log2=(9.0, 11.0), n_log10=(4.6, 5.0))
        streams = _streams(plan)
        bsk = [sf.Sketch(4, p["w"], 16, 4, p["seed"], c) for p, c in zip(plan, chunks)]
        psk = [sf.Sketch(4, p["w"], 16, 4, p["seed"], c) for p, c in zip(plan, chunks)]
        b = sf.Batch(len(plan), group_bytes=0)
        b.update([(sk, st.keys, st.ops) for sk, (st, _) in zip(bsk, streams)])
        for sk, (st, _) in zip(psk, streams):
            sk.update(st.keys, st.ops)
        assert b.sync() == sf.SF_OK
        for sk in psk:
            sk.sync()
        for i in range(len(plan)):
            assert torch.equal(bsk[i].fat, psk[i].fat) and torch.equal(bsk[i].slim, psk[i].slim), (extra, i)
        for i in (0, 9):
            p, (st, _) = plan[i], streams[i]
            o = oracle.Sketch(4, p["w"], 16, 4, p["seed"])
            o.update(st.keys.cpu().numpy(), st.ops.cpu().numpy(), S=chunks[i])
            assert np.array_equal(bsk[i].slim.cpu().numpy().view(np.uint32).reshape(o.A.shape), o.A), (extra, i)
            assert np.array_equal(bsk[i].fat.cpu().numpy().view(np.uint32).reshape(o.B.shape), o.B), (extra, i)


def test_batch_with_13_byte_keys_and_empty_items(sf):
    import torch
    sks, items, refs = [], [], []
    for i, (n, w) in enumerate([(5000, 100), (0, 64), (777, 33), (40_000, 1000)]):
        ins, dels, flows = wl.flows_with_deletes(max(n, 1), 300, 1.1, 0.1, seed=70 + i, device="cuda")
        ins = ins[:n]
        sk = sf.Sketch(4, w, 16, 13, 100 + i, 1000)
        ref = sf.Sketch(4, w, 16, 13, 100 + i, 1000)
        sks.append(sk)
        refs.append(ref)
        items.append((sk, ins, None))
        ref.insert(ins)
    b = sf.Batch(8)
    b.update(items)
    b.sync()
    for sk, ref in zip(sks, refs):
        ref.sync()
        assert torch.equal(sk.fat, ref.fat) and torch.equal(sk.slim, ref.slim)


def test_batch_with_claim_lists_in_global_memory(sf):
    """Rounds of 2.4 M slots overflow the shared-memory claim lists: the launch keeps them in the
    batch scratch instead; results still equal one call per sketch."""
    import torch
    sks, refs, items = [], [], []
    for i in range(8):
        st, _ = wl.mixed_stream(600_000, 200_000, 0.8, 0.1, 4, seed=300 + i, device="cuda")
        sk = sf.Sketch(4, 1 << 14, 16, 4, 500 + i, 300_000)
        ref = sf.Sketch(4, 1 << 14, 16, 4, 500 + i, 300_000)
        ref.update(st.keys, st.ops)
        sks.append(sk)
        refs.append(ref)
        items.append((sk, st.keys, st.ops))
    b = sf.Batch(8, max_round_slots=8 * 300_032)
    b.update(items)
    b.sync()
    for sk, ref in zip(sks, refs):
        ref.sync()
        assert torch.equal(sk.fat, ref.fat) and torch.equal(sk.slim, ref.slim)
    with pytest.raises(sf.SFError):
        small = sf.Batch(8, max_round_slots=1000)
        small.update(items)


def test_batch_mixes_sf4_and_sff_sketches(sf):
    """Sketches of both delete rules in one batched launch: each equals its own per-sketch call
    and the oracle with its rule (Sec. 3.4 SF_4, Sec. 3.5 SF_F)."""
    import torch
    plan = _plan(10, seed=21, w_log2=(6.0, 9.0), n_log10=(3.0, 4.3))
    streams = [wl.mixed_stream(p["n"], p["distinct"], p["s"], 0.3, 4, seed=p["seed"], device="cuda")[0]
               for p in plan]
    rules = ["sf4" if i % 2 else "sff" for i in range(len(plan))]
    chunks = [_chunk_for(p, 5) for p in plan]
    bsk = [sf.Sketch(4, p["w"], 16, 4, p["seed"], S, delete_rule=r) for p, S, r in zip(plan, chunks, rules)]
    b = sf.Batch(len(plan))
    b.update([(sk, st.keys, st.ops) for sk, st in zip(bsk, streams)])
    assert b.sync_status() == sf.SF_OK
    for i, (p, S, r, st) in enumerate(zip(plan, chunks, rules, streams)):
        ref = sf.Sketch(4, p["w"], 16, 4, p["seed"], S, delete_rule=r)
        ref.update(st.keys, st.ops)
        ref.sync()
        assert torch.equal(ref.fat, bsk[i].fat) and torch.equal(ref.slim, bsk[i].slim), i
        o = oracle.Sketch(4, p["w"], 16, 4, p["seed"], delete_rule=r)
        o.update(st.keys.cpu().numpy(), st.ops.cpu().numpy(), S=S)
        assert np.array_equal(bsk[i].slim.cpu().numpy().view(np.uint32).reshape(o.A.shape), o.A), (i, r)
        ref.close()
    b.close()


def _same_as_per_sketch_calls(sf, shapes, streams, bsk):
    import torch
    for (w, seed, S), (st, _), sk in zip(shapes, streams, bsk):
        ref = sf.Sketch(4, w, 16, 4, seed, S)
        ref.update(st.keys, st.ops)
        ref.sync()
        assert torch.equal(ref.fat, sk.fat) and torch.equal(ref.slim, sk.slim), (w, seed, S)
        ref.close()


@pytest.mark.parametrize("group_bytes,want_groups", [(0, 1), (8 << 20, 6), (2 << 20, 1)])
def test_launch_groups_give_the_same_sketches(sf, group_bytes, want_groups):
    """Sketches are independent, so any launch grouping gives the same sketches as one call per
    sketch.  Twelve sketches with 100,000-slot chunks (each fills the grid alone; counters
    ~3.3 MB): an 8 MiB budget packs them two per launch; a 2 MiB budget is below every sketch, so
    they share one launch; 0 is one launch."""
    shapes = [(256, 40 + i, 100_000) for i in range(12)]
    streams = [wl.mixed_stream(400_000, 3_000, 1.0, 0.1, 4, seed=seed, device="cuda") for _, seed, _ in shapes]
    bsk = [sf.Sketch(4, w, 16, 4, seed, S) for w, seed, S in shapes]
    b = sf.Batch(len(bsk), group_bytes=group_bytes, max_round_slots=12 * 100_000)
    for _ in range(2):                                    # the second call replays the captured plan
        for sk in bsk:
            sk.reset()
        b.update([(sk, st.keys, st.ops) for sk, (st, _) in zip(bsk, streams)])
    assert b.sync_status() == sf.SF_OK
    info = b.info()
    assert info["group_bytes"] == group_bytes and info["groups_last"] == want_groups
    _same_as_per_sketch_calls(sf, shapes, streams, bsk)
    b.close()


def test_underfilled_groups_join_the_shared_launch(sf):
    """Small sketches whose groups would leave most of the grid idle all run in one launch, with
    the same results."""
    plan = _plan(30, seed=11)
    streams = _streams(plan)
    shapes = [(p["w"], p["seed"], _chunk_for(p, 6)) for p in plan]
    bsk = [sf.Sketch(4, w, 16, 4, seed, S) for w, seed, S in shapes]
    b = sf.Batch(len(bsk), group_bytes=150_000)
    b.update([(sk, st.keys, st.ops) for sk, (st, _) in zip(bsk, streams)])
    assert b.sync_status() == sf.SF_OK
    assert b.info()["groups_last"] == 1
    _same_as_per_sketch_calls(sf, shapes, streams, bsk)
    b.close()


def test_dictionary_arena_splits_launches_and_gives_the_same_sketches(sf):
    """SF_FLAG_SHARED_DICT sketches take their chunk dictionaries from the batch's arena, per launch:
    twelve sketches with 100,000-slot chunks (32 MiB dictionaries) in one launch (group budget 0)
    with an 80 MiB arena run as six launches of two, and small sketches of the single-iteration
    kernel with an arena of three dictionaries split the same way; every sketch equals one
    sf_update_batch call per sketch, on the second call (graph replay) as on the first.  A sketch
    whose dictionary exceeds the arena is SF_ERR_OOM; a flagged sketch with neither an arena nor
    its own dictionary is SF_ERR_INVALID."""
    shapes = [(256, 40 + i, 100_000) for i in range(12)]
    streams = [wl.mixed_stream(400_000, 3_000, 1.0, 0.1, 4, seed=seed, device="cuda") for _, seed, _ in shapes]
    bsk = [sf.Sketch(4, w, 16, 4, seed, S, shared_dict=True) for w, seed, S in shapes]
    dict_bytes = sf.dictionary_bytes(4, 256, 16, 4, 0, 100_000)
    assert dict_bytes == 32 << 20
    b = sf.Batch(len(bsk), group_bytes=0, max_round_slots=12 * 100_000, dict_arena_bytes=80 << 20)
    for _ in range(2):
        for sk in bsk:
            sk.reset()
        b.update([(sk, st.keys, st.ops) for sk, (st, _) in zip(bsk, streams)])
    assert b.sync_status() == sf.SF_OK
    assert b.info()["groups_last"] == 6
    _same_as_per_sketch_calls(sf, shapes, streams, bsk)
    b.close()

    plan = _plan(30, seed=13)
    pstreams = _streams(plan)
    pshapes = [(p["w"], p["seed"], _chunk_for(p, 6)) for p in plan]
    psk = [sf.Sketch(4, w, 16, 4, seed, S, shared_dict=True) for w, seed, S in pshapes]
    needs = [sf.dictionary_bytes(4, w, 16, 4, seed, S) for w, seed, S in pshapes]
    arena = 3 * max(needs)
    want, used = 1, 0                 # launches of the greedy in-order split
    for nb in needs:
        if used and used + nb > arena:
            want, used = want + 1, 0
        used += nb
    assert want > 1
    b2 = sf.Batch(len(psk), group_bytes=0, dict_arena_bytes=arena)
    b2.update([(sk, st.keys, st.ops) for sk, (st, _) in zip(psk, pstreams)])
    assert b2.sync_status() == sf.SF_OK
    assert b2.info()["groups_last"] == want
    _same_as_per_sketch_calls(sf, pshapes, pstreams, psk)
    b2.close()

    small = sf.Batch(1, dict_arena_bytes=dict_bytes // 2, max_round_slots=100_000)
    with pytest.raises(sf.SFError) as ei:
        small.update([(bsk[0], streams[0][0].keys, streams[0][0].ops)])
    assert ei.value.status == sf.SF_ERR_OOM
    small.close()
    bare = sf.Batch(1, max_round_slots=100_000)
    with pytest.raises(sf.SFError) as ei:
        bare.update([(bsk[0], streams[0][0].keys, streams[0][0].ops)])
    assert ei.value.status == sf.SF_ERR_INVALID
    bare.close()


def test_shared_dictionary_for_standalone_updates(sf):
    """Two SF_FLAG_SHARED_DICT sketches (13-byte keys, chunk 4,096; u32 keys, chunk 100,000) whose
    calls run one after another on one stream share one dictionary buffer (sf_set_dictionary) and
    equal sketches that own theirs.  Without a dictionary a flagged sketch refuses an update; too
    small a buffer is refused."""
    import torch
    ins, dels, _ = wl.flows_with_deletes(200_000, 20_000, 1.0, 0.1, seed=81)
    st4, _ = wl.mixed_stream(300_000, 20_000, 1.2, 0.2, 4, seed=82, device="cuda")
    a1, a2 = sf.Sketch(4, 3001, 16, 13, 5, 4096), sf.Sketch(4, 777, 8, 4, 6, 100_000)
    b1 = sf.Sketch(4, 3001, 16, 13, 5, 4096, shared_dict=True)
    b2 = sf.Sketch(4, 777, 8, 4, 6, 100_000, shared_dict=True)
    with pytest.raises(sf.SFError) as ei:
        b1.insert(ins.cuda())
    assert ei.value.status == sf.SF_ERR_INVALID
    need = max(sf.dictionary_bytes(4, 3001, 16, 13, 5, 4096), sf.dictionary_bytes(4, 777, 8, 4, 6, 100_000))
    with pytest.raises(sf.SFError) as ei:
        b2.set_dictionary(torch.empty(need // 2, dtype=torch.uint8, device="cuda"))
    assert ei.value.status == sf.SF_ERR_INVALID
    shared = torch.empty(need, dtype=torch.uint8, device="cuda")
    b1.set_dictionary(shared)
    b2.set_dictionary(shared)
    for a, b, call in ((a1, b1, lambda s: s.insert(ins.cuda())), (a2, b2, lambda s: s.update(st4.keys, st4.ops)),
                       (a1, b1, lambda s: s.delete(dels.cuda()))):
        call(a)
        call(b)
    for s in (a1, a2, b1, b2):
        assert s.sync_status() == sf.SF_OK
    assert torch.equal(a1.fat, b1.fat) and torch.equal(a1.slim, b1.slim)
    assert torch.equal(a2.fat, b2.fat) and torch.equal(a2.slim, b2.slim)


def test_dictionary_arena_with_13_byte_keys_and_deletes_and_a_pipelined_sketch(sf):
    """The arena with 13-byte flow keys and mixed insert/delete operations (single-iteration and
    multi-iteration chunk sizes in one batch, launches split by the arena), and a flagged sketch
    updated from pinned host keys through an sf_pipeline with a dictionary of its own: every
    sketch equals the same sketch that owns its dictionary."""
    import torch
    shapes = [(3001, 90 + i, S) for i, S in enumerate((4096, 65536, 100_000, 2048, 70_000, 30_000))]
    streams = []
    for w, seed, S in shapes:
        ins, dels, _ = wl.flows_with_deletes(150_000, 20_000, 1.0, 0.15, seed=seed, device="cuda")
        keys = torch.cat([ins, dels]).contiguous()
        ops = torch.cat([torch.ones(ins.shape[0], dtype=torch.int8, device="cuda"),
                         -torch.ones(dels.shape[0], dtype=torch.int8, device="cuda")]).contiguous()
        streams.append((keys, ops))
    flagged = [sf.Sketch(4, w, 16, 13, seed, S, shared_dict=True) for w, seed, S in shapes]
    arena = 2 * max(sf.dictionary_bytes(4, w, 16, 13, seed, S) for w, seed, S in shapes)
    b = sf.Batch(len(flagged), group_bytes=0, max_round_slots=sum(S for _, _, S in shapes) + 32 * len(shapes),
                 dict_arena_bytes=arena)
    b.update([(sk, k, o) for sk, (k, o) in zip(flagged, streams)])
    assert b.sync_status() == sf.SF_OK
    assert b.info()["groups_last"] >= 3
    for (w, seed, S), (k, o), sk in zip(shapes, streams, flagged):
        ref = sf.Sketch(4, w, 16, 13, seed, S)
        ref.update(k, o)
        assert ref.sync_status() == sf.SF_OK
        assert torch.equal(ref.fat, sk.fat) and torch.equal(ref.slim, sk.slim), (w, seed, S)
        ref.close()
    b.close()

    w, seed, S = shapes[2]
    k, o = streams[2]
    ref = sf.Sketch(4, w, 16, 13, seed, S)
    ref.update(k, o)
    p_sk = sf.Sketch(4, w, 16, 13, seed, S, shared_dict=True)
    p_sk.set_dictionary(torch.empty(sf.dictionary_bytes(4, w, 16, 13, seed, S), dtype=torch.uint8, device="cuda"))
    pipe = sf.Pipeline(staging_bytes=2 * (S * 14 + 32))
    p_sk.update_through(pipe, k.cpu().pin_memory(), o.cpu().pin_memory())
    assert ref.sync_status() == sf.SF_OK and p_sk.sync_status() == sf.SF_OK
    assert torch.equal(ref.fat, p_sk.fat) and torch.equal(ref.slim, p_sk.slim)
    pipe.close()
