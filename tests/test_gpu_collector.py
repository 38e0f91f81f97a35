"""Collector serving loop (sfc_*): answers equal sf_query_batch on the same Slim whether a request
runs alone or inside a mix of concurrent requests; queries bind to the sketch version current at
submit; uploads are admitted by the memory budget."""
import threading

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


def _make_slim(sf, w, seed, n_updates, key_bytes=4):
    import torch
    sk = sf.Sketch(4, w, 16, key_bytes, seed, 512)
    st, ids = wl.mixed_stream(n_updates, max(64, 4 * w), 1.0, 0.1, key_bytes, seed=seed, device="cuda")
    sk.update(st.keys, st.ops)
    slim, hdr = sk.export_slim()
    sk.sync()
    return slim, hdr, ids


def _reference(sf, slim, hdr, keys_np):
    import torch
    return sf.query(slim, hdr, torch.from_numpy(keys_np).cuda()).cpu().numpy().view(np.uint32)


def test_answers_alone_and_in_the_mix(sf):
    import torch
    rng = np.random.default_rng(3)
    slims = [_make_slim(sf, int(w), 10 + i, 20_000) for i, w in enumerate([1024, 3000, 65536, 4096, 777])]
    col = sf.Collector(budget_bytes=64 << 20, max_sketches=16, n_streams=4, max_batch_keys=1 << 16, max_wait_us=100)
    for i, (slim, hdr, _) in enumerate(slims):
        assert col.upload(i, slim, hdr) == sf.SF_OK
    reqs = []
    for q in range(400):
        i = int(rng.integers(len(slims)))
        n = int(2 ** rng.uniform(0, 14))
        ids = slims[i][2].cpu().numpy()
        keys = np.ascontiguousarray(ids[rng.integers(0, len(ids), n)])
        reqs.append((i, keys, _reference(sf, slims[i][0], slims[i][1], keys)))
    # alone: one request at a time
    for i, keys, want in reqs[:40]:
        out = np.zeros(len(want), np.uint32)
        t = col.submit(i, keys, out)
        assert col.wait(t) == sf.SF_OK
        assert np.array_equal(out, want)
    # in the mix: 4 threads submitting concurrently, each waiting later
    outs = [None] * len(reqs)

    def client(lo, hi):
        tickets = []
        for r in range(lo, hi):
            i, keys, want = reqs[r]
            out = np.zeros(len(want), np.uint32)
            outs[r] = out
            tickets.append(col.submit(i, keys, out))
        for t in tickets:
            assert col.wait(t) == sf.SF_OK

    th = [threading.Thread(target=client, args=(k * 100, (k + 1) * 100)) for k in range(4)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    for r, (i, keys, want) in enumerate(reqs):
        assert np.array_equal(outs[r], want), r
    st = col.stats()
    assert st["requests"] == 440 and st["batches"] < 440 and st["p99_us"] >= st["p50_us"] > 0
    col.close()


def test_queries_bind_to_the_version_current_at_submit(sf):
    import torch
    a, ha, ids = _make_slim(sf, 2048, 21, 30_000)
    b, hb, _ = _make_slim(sf, 2048, 21, 60_000)  # same sketch shape, more updates: a newer version
    col = sf.Collector(budget_bytes=1 << 20, max_sketches=2, n_streams=2, max_wait_us=2000)
    assert col.upload(0, a, ha) == sf.SF_OK
    keys = np.ascontiguousarray(ids.cpu().numpy()[:5000])
    want_a, want_b = _reference(sf, a, ha, keys), _reference(sf, b, hb, keys)
    assert not np.array_equal(want_a, want_b)
    out1 = np.zeros(len(keys), np.uint32)
    t1 = col.submit(0, keys, out1)          # bound to version a
    assert col.upload(0, b, hb) == sf.SF_OK  # replace in place
    out2 = np.zeros(len(keys), np.uint32)
    t2 = col.submit(0, keys, out2)          # bound to version b
    assert col.wait(t1) == sf.SF_OK and col.wait(t2) == sf.SF_OK
    assert np.array_equal(out1, want_a) and np.array_equal(out2, want_b)
    col.close()


def test_budget_admission(sf):
    import torch
    s1, h1, _ = _make_slim(sf, 16384, 31, 5000)   # 256 KiB each
    s2, h2, _ = _make_slim(sf, 16384, 32, 5000)
    s3, h3, _ = _make_slim(sf, 16384, 33, 5000)
    col = sf.Collector(budget_bytes=600 * 1024, max_sketches=4, n_streams=1)
    assert col.upload(0, s1, h1) == sf.SF_OK
    assert col.upload(1, s2, h2) == sf.SF_OK
    assert col.upload(2, s3, h3) == sf.SF_ERR_BUDGET
    assert col.evict(0) == sf.SF_OK
    assert col.upload(2, s3, h3) == sf.SF_OK
    st = col.stats()
    assert st["rejected_uploads"] == 1 and st["uploads"] == 3 and st["arena_used_bytes"] == 2 * 256 * 1024
    bad = sf.SlimHeader(0xDEAD, 1, 4, 16384, 4, 1, 0)
    assert col.upload(3, s1, bad) == sf.SF_ERR_VERSION
    col.close()
