"""Collector serving loop (sfc_*): every answer equals the CPU oracle's point query (Sec. 3.1:
the minimum of the key's d Slim counters) on the exact Slim contents the request is bound to,
whether a request runs alone or inside a mix of concurrent requests; queries bind to the sketch
version current at submit; uploads are admitted by the memory budget."""
import threading

import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu


def _make_slim(sf, w, seed, n_updates, key_bytes=4):
    """A Slim exported from a GPU sketch fed a turnstile stream; returns (slim, header, distinct keys)."""
    sk = sf.Sketch(4, w, 16, key_bytes, seed, 512)
    if key_bytes == 13:
        ins, dels, ids = wl.flows_with_deletes(n_updates, max(64, 4 * w), 1.0, 0.1, seed=seed, device="cuda")
        sk.insert(ins)
        sk.delete(dels)
    else:
        st, ids = wl.mixed_stream(n_updates, max(64, 4 * w), 1.0, 0.1, key_bytes, seed=seed, device="cuda")
        sk.update(st.keys, st.ops)
    slim, hdr = sk.export_slim()
    sk.sync()
    return slim, hdr, ids


def _reference(sf, slim, hdr, keys_np):
    """The oracle's query (Sec. 3.1) on these Slim counters, read back from the device."""
    o = oracle.Sketch(hdr.d, hdr.w, 1, hdr.key_bytes, hdr.seed)
    o.A[...] = slim.cpu().numpy().view(np.uint32).reshape(hdr.d, hdr.w)
    return o.query(keys_np)


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


def test_answers_match_the_oracle_across_key_widths_and_replacement(sf):
    """Mixed key widths (4, 8, 13 bytes) and widths that are not powers of two, requests of
    1..16,384 keys from four threads, then a replace-in-place upload with requests bound to the
    old and the new version in flight together: every answer equals the oracle's."""
    rng = np.random.default_rng(17)
    shapes = [(1024, 4), (3000, 8), (777, 13), (65536, 13), (12288, 4), (40000, 8)]
    slims = [_make_slim(sf, w, 50 + i, 30_000, kb) for i, (w, kb) in enumerate(shapes)]
    col = sf.Collector(budget_bytes=32 << 20, max_sketches=8, n_streams=4, max_batch_keys=1 << 15, max_wait_us=200)
    for i, (slim, hdr, _) in enumerate(slims):
        assert col.upload(i, slim, hdr) == sf.SF_OK

    def request(i, n, version):
        slim, hdr, ids = version
        ids = ids.cpu().numpy()
        present = ids[rng.integers(0, len(ids), n - n // 5)]
        absent = rng.integers(0, 256, (n // 5, hdr.key_bytes), dtype=np.uint8)
        keys = np.ascontiguousarray(np.concatenate([present, absent])[rng.permutation(n)])
        return i, keys, _reference(sf, slim, hdr, keys)

    reqs = [request(int(i), int(2 ** rng.uniform(0, 14)), slims[int(i)]) for i in rng.integers(0, len(slims), 240)]
    outs = [None] * len(reqs)

    def client(lo, hi):
        tickets = []
        for r in range(lo, hi):
            i, keys, want = reqs[r]
            outs[r] = np.zeros(len(want), np.uint32)
            tickets.append(col.submit(i, keys, outs[r]))
        for t in tickets:
            assert col.wait(t) == sf.SF_OK

    th = [threading.Thread(target=client, args=(k * 60, (k + 1) * 60)) for k in range(4)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    for r, (i, keys, want) in enumerate(reqs):
        assert np.array_equal(outs[r], want), (r, shapes[i])

    # replace sketch 3 (13-byte keys, w = 65,536) in place while requests on the old version run
    newer = _make_slim(sf, 65536, 53, 90_000, 13)
    old_reqs = [request(3, 4096, slims[3]) for _ in range(6)]
    old_out = [np.zeros(4096, np.uint32) for _ in old_reqs]
    old_t = [col.submit(3, k, o) for (_, k, _), o in zip(old_reqs, old_out)]
    assert col.upload(3, newer[0], newer[1]) == sf.SF_OK
    new_reqs = [request(3, 4096, newer) for _ in range(6)]
    new_out = [np.zeros(4096, np.uint32) for _ in new_reqs]
    new_t = [col.submit(3, k, o) for (_, k, _), o in zip(new_reqs, new_out)]
    for t in old_t + new_t:
        assert col.wait(t) == sf.SF_OK
    for (_, _, want), got in zip(old_reqs + new_reqs, old_out + new_out):
        assert np.array_equal(got, want)
    col.close()


def test_slim_queries_of_the_library_match_the_oracle(sf):
    """sf_query_batch (the one-Slim query kernel) on the same Slims, for every key width."""
    import torch
    for i, (w, kb) in enumerate([(1000, 4), (5000, 8), (777, 13)]):
        slim, hdr, ids = _make_slim(sf, w, 70 + i, 20_000, kb)
        keys = ids.cpu().numpy()
        got = sf.query(slim, hdr, torch.from_numpy(keys).cuda()).cpu().numpy().view(np.uint32)
        assert np.array_equal(got, _reference(sf, slim, hdr, keys))
