"""The measured configurations at their full sizes, on the GPU, against the CPU oracle.

- insert-only u32 keys with chunk 1 (the paper's one-at-a-time rule): every counter and query;
- 13-byte flows, Zipf sweep, 32 M inserts + 3.2 M deletes, chunk 65,536: every counter and
  every query for each s (the oracle runs the same chunked semantics);
- 1,024 uneven sketches in one batched launch: batched == one call per sketch for all, and
  sampled sketches == the oracle;
- 10^9 u64 keys, 80/20 turnstile, 1 GiB Fat, chunk 2^20: the first two chunks counter by counter
  against the oracle, then properties of the full run (Fat row sums, no under-estimation
  against exact counts, Slim <= bucket maximum).
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


def test_insert_only_chunk_one_full_size(sf):
    import torch
    keys, ids = wl.insert_only_u32(100_000, 10_000, 1.0, seed=1)
    d, w, z = 4, 4096, 16
    g = sf.Sketch(d, w, z, 4, 1, 1)
    g.insert(keys.cuda())
    slim, hdr = g.export_slim()
    est = sf.query(slim, hdr, ids.cuda())
    g.sync()
    o = oracle.Sketch(d, w, z, 4, 1)
    o.update(keys.numpy(), np.ones(len(keys), np.int8), S=None)   # SEQ: the paper's rule
    assert np.array_equal(_u32(g.fat).reshape(o.B.shape), o.B)
    assert np.array_equal(_u32(slim).reshape(o.A.shape), o.A)
    assert np.array_equal(_u32(est), o.query(ids.numpy()))


@pytest.mark.parametrize("s", wl.ZIPF_SWEEP)
def test_flows_full_size(sf, s):
    import torch
    idx = wl.ZIPF_SWEEP.index(s)
    ins, dels, flows = wl.flows_with_deletes(32_000_000, 1_000_000, s, 0.1, seed=2 + idx, device="cuda")
    d, w, z, S = 4, 1 << 18, 16, 65536
    g = sf.Sketch(d, w, z, 13, 2, S)
    g.insert(ins)
    g.delete(dels)
    slim, hdr = g.export_slim()
    est = sf.query(slim, hdr, flows)
    g.sync()
    o = oracle.Sketch(d, w, z, 13, 2)
    o.update(ins.cpu().numpy(), np.ones(ins.shape[0], np.int8), S=S)
    o.update(dels.cpu().numpy(), -np.ones(dels.shape[0], np.int8), S=S)
    assert np.array_equal(_u32(g.fat).reshape(o.B.shape), o.B)
    assert np.array_equal(_u32(slim).reshape(o.A.shape), o.A)
    assert np.array_equal(_u32(est), o.query(flows.cpu().numpy()))


def test_many_sketches_full_size(sf):
    import torch
    from paper_1701_04148_gb300 import autotune
    plan = wl.many_sketch_plan(1024, seed=3)
    streams = []
    for p in plan:
        st, _ = wl.mixed_stream(p["n"], p["distinct"], p["s"], 0.1, 4, seed=p["seed"], device="cuda")
        streams.append(st)
    chunks = autotune.chunk_sizes([p["n"] for p in plan], 256)
    bsk = [sf.Sketch(4, p["w"], 16, 4, p["seed"], S) for p, S in zip(plan, chunks)]
    b = sf.Batch(len(bsk), max_round_slots=sum((c + 31) // 32 * 32 for c in chunks))
    b.update([(sk, st.keys, st.ops) for sk, st in zip(bsk, streams)])
    assert b.sync_status() == sf.SF_OK
    for i, (p, S, st) in enumerate(zip(plan, chunks, streams)):
        ref = sf.Sketch(4, p["w"], 16, 4, p["seed"], S)
        ref.update(st.keys, st.ops)
        ref.sync()
        assert torch.equal(ref.fat, bsk[i].fat) and torch.equal(ref.slim, bsk[i].slim), i
        ref.close()
    small = sorted(range(len(plan)), key=lambda i: plan[i]["n"])[:: len(plan) // 6][:6]
    for i in small:
        p, S, st = plan[i], chunks[i], streams[i]
        o = oracle.Sketch(4, p["w"], 16, 4, p["seed"])
        o.update(st.keys.cpu().numpy(), st.ops.cpu().numpy(), S=S)
        assert np.array_equal(_u32(bsk[i].fat).reshape(o.B.shape), o.B), i
        assert np.array_equal(_u32(bsk[i].slim).reshape(o.A.shape), o.A), i


def test_out_of_l2_stress_full_size(sf):
    import torch
    d, w, z, S = 4, 1 << 22, 16, 1 << 20
    st, ids = wl.mixed_stream(1_000_000_000, 1 << 26, 1.2, 0.2, 8, seed=5, device="cuda")
    keys, ops = st.keys, st.ops
    n = keys.shape[0]
    g = sf.Sketch(d, w, z, 8, 5, S)
    # the first two chunks, counter by counter against the oracle
    pre = 2 * S
    g.update(keys[:pre], ops[:pre])
    g.sync()
    o = oracle.Sketch(d, w, z, 8, 5)
    o.update(keys[:pre].cpu().numpy(), ops[:pre].cpu().numpy(), S=S)
    assert np.array_equal(_u32(g.fat).reshape(o.B.shape), o.B)
    assert np.array_equal(_u32(g.slim).reshape(o.A.shape), o.A)
    del o
    # the rest of the stream in one more call (a new call starts a new chunk)
    g.update(keys[pre:], ops[pre:])
    assert g.sync_status() == sf.SF_OK
    net = int(ops.to(torch.int64).sum())
    fat = g.fat.view(d, w * z).to(torch.int64) & 0xFFFFFFFF
    assert all(int(fat[i].sum()) == net for i in range(d))
    A = g.slim.view(d, w).to(torch.int64) & 0xFFFFFFFF
    assert bool((A <= fat.view(d, w, z).max(dim=2).values).all())
    # exact net frequencies by sorting the stream; queries: half present keys (distinct keys of the
    # stream), half random 64-bit ids (absent with overwhelming probability)
    kid = keys.view(torch.int64).reshape(-1)
    skeys, order = torch.sort(kid)
    sops = ops.to(torch.int64)[order]
    del order
    uniq, inv = torch.unique_consecutive(skeys, return_inverse=True)
    freq = torch.zeros(uniq.numel(), dtype=torch.int64, device="cuda").index_add_(0, inv, sops)
    del skeys, inv, sops
    gq = torch.Generator(device="cuda").manual_seed(77)
    q_present = uniq[torch.randint(0, uniq.numel(), (1 << 23,), device="cuda", generator=gq)]
    q_absent = torch.randint(-(1 << 62), 1 << 62, (1 << 23,), device="cuda", generator=gq)
    q = torch.cat([q_present, q_absent])
    slim, hdr = g.export_slim()
    est = sf.query(slim, hdr, q.view(torch.uint8).reshape(-1, 8).contiguous()).to(torch.int64) & 0xFFFFFFFF
    pos = torch.searchsorted(uniq, q).clamp(max=uniq.numel() - 1)
    f = torch.where(uniq[pos] == q, freq[pos], torch.zeros_like(q))
    assert bool((est >= f).all()), "under-estimation"
    assert int(f[: 1 << 23].gt(0).sum()) > (1 << 22)
