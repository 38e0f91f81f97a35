"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: published vectors,
the paper's worked example, its theorems, closed forms, invariants, and brute force
against a separately written literal transcription of the paper's rules.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import Sketch, explicit_indices

GOLD = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1


# ---------------------------------------------------------------------------------------
# hash reading: SplitMix64 (Steele, Lea, Flood 2014) + multiply-shift reduction (Lemire 2019)
# ---------------------------------------------------------------------------------------

def test_splitmix64_published_vectors():
    g = json.load(open(os.path.join(GOLD, "splitmix64_vectors.json")))
    for v in g["vectors"]:
        if "outputs_hex" in v:
            want = [int(x, 16) for x in v["outputs_hex"]]
        else:
            want = [int(x) for x in v["outputs_dec"]]
        assert oracle.splitmix64_sequence(v["seed"], len(want)) == want


def _unxorshift(y, k):
    r = y
    for _ in range(64 // k + 1):
        r = y ^ (r >> k)
    return r & M64


def _inverse_mix64(y):
    y = _unxorshift(y, 31)
    y = (y * pow(0x94D049BB133111EB, -1, 1 << 64)) & M64
    y = _unxorshift(y, 27)
    y = (y * pow(0xBF58476D1CE4E5B9, -1, 1 << 64)) & M64
    y = _unxorshift(y, 30)
    return y


def test_mix64_inverts_with_the_published_constants():
    rng = np.random.default_rng(7)
    for x in [0, 1, M64, 0x0123456789ABCDEF] + [int(v) for v in rng.integers(0, 2**63, 200)]:
        assert _inverse_mix64(oracle.mix64(x)) == x


def test_row_seeds_are_the_splitmix64_sequence():
    for seed in (0, 1234567, 2**63 + 5):
        assert [int(s) for s in oracle.row_seeds(seed, 6)] == oracle.splitmix64_sequence(seed, 6)


@pytest.mark.parametrize("w,z", [(4096, 16), (1 << 18, 16), (1, 1), (2, 2)])
def test_power_of_two_reduction_takes_the_top_bits(w, z):
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 2**32, 500, dtype=np.uint64).astype(np.uint32)
    seed = 99
    h, f = oracle.index_keys(keys.view(np.uint8).reshape(-1, 4), seed, 3, w, z)
    rs = oracle.row_seeds(seed, 3)
    kw, kz = w.bit_length() - 1, z.bit_length() - 1
    for t in range(len(keys)):
        for i in range(3):
            H = oracle.mix64(int(keys[t]) ^ int(rs[i]))
            assert h[t, i] == ((H >> 32) >> (32 - kw) if kw else 0)
            assert f[t, i] == ((H & 0xFFFFFFFF) >> (32 - kz) if kz else 0)


def test_general_width_reduction_is_uniform_and_in_range():
    rng = np.random.default_rng(11)
    n, w, z = 200_000, 1000, 16
    keys = rng.integers(0, 2**63, n, dtype=np.uint64)
    h, f = oracle.index_keys(keys.view(np.uint8).reshape(-1, 8), 5, 2, w, z)
    assert h.max() < w and f.max() < z
    for col, m in ((h[:, 0], w), (h[:, 1], w), (f[:, 0], z)):
        cnt = np.bincount(col, minlength=m)
        chi2 = float(((cnt - n / m) ** 2 / (n / m)).sum())
        # chi-square with m-1 dof: mean m-1, sd sqrt(2(m-1)); allow 5 sd
        assert abs(chi2 - (m - 1)) < 5 * np.sqrt(2 * (m - 1))


def test_13_byte_keys_use_all_bytes():
    rng = np.random.default_rng(5)
    k = rng.integers(0, 256, (1, 13), dtype=np.uint8)
    h0, _ = oracle.index_keys(k, 1, 4, 1 << 20, 16)
    for b in range(13):
        k2 = k.copy()
        k2[0, b] ^= 1
        h2, _ = oracle.index_keys(k2, 1, 4, 1 << 20, 16)
        assert not np.array_equal(h0, h2), f"byte {b} does not reach the hash"


W_MAX = 0xFFFFFFFF


def _published_1234567():
    g = json.load(open(os.path.join(GOLD, "splitmix64_vectors.json")))
    v = next(v for v in g["vectors"] if v["seed"] == 1234567)
    return [int(x) for x in v["outputs_dec"]]


def _le(row) -> int:
    return sum(int(b) << (8 * i) for i, b in enumerate(row))


def _key8(x0: int) -> np.ndarray:
    return np.array([[(x0 >> (8 * b)) & 0xFF for b in range(8)]], dtype=np.uint8)


def _hash_read_back(keys: np.ndarray, seed: int, d: int):
    """H_i of every key, read back from the oracle's indices at w = z = 2^32 - 1, where the
    reduction returns max(x - 1, 0) of each 32-bit half (pinned by the partition test below).
    Keys with a half in {0, 1} (ambiguous; probability 2^-31 each) come back as None."""
    h, f = oracle.index_keys(keys, seed, d, W_MAX, W_MAX)
    out = []
    for t in range(len(keys)):
        row = []
        for i in range(d):
            hi, lo = int(h[t, i]), int(f[t, i])
            row.append(None if hi == 0 or lo == 0 else ((hi + 1) << 32) | (lo + 1))
        out.append(row)
    return out


@pytest.mark.parametrize("w", [3, 7, 1000, 40_000, 65_537, 393_217, 2**31 - 1, W_MAX])
def test_multiply_shift_partitions_the_32_bit_range_in_order(w):
    """Multiply-shift range reduction (Lemire, ACM TOMACS 2019) splits [0, 2^32) into w contiguous
    runs in increasing order; run j starts at ceil(j * 2^32 / w).  So the first input of run j maps
    to j and the input just before it to j - 1.  Checked at run starts spread over the range, for
    the bucket h (top half of H) and, with z = w, the slot f (low half), on 8-byte keys built to
    hash to chosen H through the inverse of mix64 derived above and the row seed (the first
    SplitMix64 output of the seed, pinned by the published vectors)."""
    seed = 1234567
    s0 = _published_1234567()[0]
    rng = np.random.default_rng(w % 1000003)
    js = sorted({1, 2, w // 3, w // 2, w - 1} | {int(x) for x in rng.integers(1, w, 40)})
    targets, want = [], []
    for j in js:
        t = (j * 2**32 + w - 1) // w  # first input of run j
        targets += [(t << 32) | t, ((t - 1) << 32) | (t - 1)]
        want += [j, j - 1]
    targets += [0, M64]
    want += [0, w - 1]
    keys = np.concatenate([_key8(_inverse_mix64(H) ^ s0) for H in targets])
    h, f = oracle.index_keys(keys, seed, 1, w, w)
    assert [int(x) for x in h[:, 0]] == want
    assert [int(x) for x in f[:, 0]] == want


@pytest.mark.parametrize("kb", [1, 3, 4, 8])
def test_short_keys_hash_as_one_mix_of_the_key_xor_the_row_seed(kb):
    """Keys of at most 8 bytes: H_i = mix64(x0 ^ s_i), x0 = the key bytes little-endian.  So
    mix64^-1(H_i) ^ x0 is the same for every key and equals s_i, the i-th published SplitMix64
    output of the sketch seed (five rows, five published outputs)."""
    rng = np.random.default_rng(kb)
    keys = rng.integers(0, 256, (300, kb), dtype=np.uint8)
    pub = _published_1234567()
    H = _hash_read_back(keys, 1234567, 5)
    seen = 0
    for t in range(len(keys)):
        for i in range(5):
            if H[t][i] is not None:
                assert _inverse_mix64(H[t][i]) ^ _le(keys[t]) == pub[i], (t, i)
                seen += 1
    assert seen > 1400


@pytest.mark.parametrize("kb", [9, 13, 15])
def test_long_keys_fold_the_second_word_in_after_the_first_mix(kb):
    """Keys of 9..15 bytes: H_i = mix64(mix64(x0 ^ s_i) ^ x1), x0 = bytes 0..7 and x1 = bytes 8..
    little-endian.  So mix64^-1(H_i) ^ x1 does not depend on the tail and equals the hash of the
    8-byte key x0 alone (both hashes read back from the oracle): a swapped or reordered word, a
    big-endian tail or a dropped fold all break it."""
    rng = np.random.default_rng(100 + kb)
    d = 4
    for _ in range(20):
        head = rng.integers(0, 256, (1, 8), dtype=np.uint8)
        tails = rng.integers(0, 256, (12, kb - 8), dtype=np.uint8)
        tails[0] = 0
        keys = np.concatenate([np.repeat(head, len(tails), 0), tails], axis=1)
        H8 = _hash_read_back(head, 77, d)[0]
        H = _hash_read_back(keys, 77, d)
        for t in range(len(keys)):
            for i in range(d):
                if H[t][i] is None or H8[i] is None:
                    continue
                assert _inverse_mix64(H[t][i]) ^ _le(tails[t]) == H8[i], (t, i)


# ---------------------------------------------------------------------------------------
# the worked example of Sec. 3.2 (Fig. 3)
# ---------------------------------------------------------------------------------------

def _worked_example_run(semantics, fchoice):
    g = json.load(open(os.path.join(GOLD, "worked_example_fig3.json")))
    d, w, z = g["d"], g["w"], g["z"]
    table = np.zeros((2, d, 2), dtype=np.uint32)
    for k, name in enumerate(("e1", "e2")):
        table[k, :, 0] = g["keys"][name]["h"]
        table[k, :, 1] = fchoice[k]
    sk = Sketch(d, w, z)
    ids = np.array([0, 1], dtype=np.uint32)
    h, f, ident = explicit_indices(table, ids)
    if semantics == "seq":
        sk.seq_apply(h, f, np.array([1, 1], np.int8))
    else:
        sk.chunk_apply(h, f, np.array([1, 1], np.int8), 1, ident)
    after_ins = sk.A.copy()
    h, f, ident = explicit_indices(table, np.array([0], np.uint32))
    if semantics == "seq":
        sk.seq_apply(h, f, np.array([-1], np.int8))
    else:
        sk.chunk_apply(h, f, np.array([-1], np.int8), 1, ident)
    hq, _, _ = explicit_indices(table, ids)
    return g, after_ins, sk.A.copy(), sk.query_idx(hq)


@pytest.mark.parametrize("semantics", ["seq", "chunk1"])
def test_worked_example_sec32(semantics):
    g = json.load(open(os.path.join(GOLD, "worked_example_fig3.json")))
    for fchoice in g["fat_slot_choices"]:
        _, after_ins, after_del, q = _worked_example_run(semantics, fchoice)
        assert after_ins.tolist() == g["after_inserts_printed_by_paper"]["A"]
        assert after_del.tolist() == g["after_delete_e1_by_SF_F_rule"]["A"]
        assert q.tolist() == [g["after_delete_e1_by_SF_F_rule"]["query"]["e1"],
                              g["after_delete_e1_by_SF_F_rule"]["query"]["e2"]]


# ---------------------------------------------------------------------------------------
# a literal transcription of the paper's one-at-a-time rules, written separately (pure Python)
# ---------------------------------------------------------------------------------------

def py_literal_seq(d, w, z, idx_of_key, stream):
    A = [[0] * w for _ in range(d)]
    B = [[[0] * z for _ in range(w)] for _ in range(d)]
    for key, op in stream:
        hs, fs = idx_of_key[key]
        if op > 0:  # Sec. 3.4 insertion (SF_F inserts like SF_4)
            for i in range(d):
                B[i][hs[i]][fs[i]] += 1
            bmin = min(B[i][hs[i]][fs[i]] for i in range(d))
            smallest = min(A[i][hs[i]] for i in range(d))
            if smallest < bmin:
                for l in range(d):
                    if A[l][hs[l]] == smallest:
                        A[l][hs[l]] += 1
        else:  # Sec. 3.5 deletion
            for i in range(d):
                before = max(B[i][hs[i]])
                B[i][hs[i]][fs[i]] -= 1
                after = max(B[i][hs[i]])
                if after != before and A[i][hs[i]] > after:
                    A[i][hs[i]] = after
    return np.array(A, dtype=np.uint32), np.array(B, dtype=np.uint32)


def _tiny_streams(n_keys, max_len):
    """All strict-turnstile streams over n_keys keys up to max_len updates."""
    out = []

    def rec(prefix, counts):
        out.append(list(prefix))
        if len(prefix) == max_len:
            return
        for k in range(n_keys):
            rec(prefix + [(k, 1)], counts[:k] + (counts[k] + 1,) + counts[k + 1:])
            if counts[k] > 0:
                rec(prefix + [(k, -1)], counts[:k] + (counts[k] - 1,) + counts[k + 1:])

    rec([], (0,) * n_keys)
    return out


@pytest.mark.parametrize("layout", [
    # (h per key per row, f per key per row) for d=2, w=2, z=2, 3 keys
    ([[0, 0], [0, 1], [1, 1]], [[0, 1], [1, 0], [0, 0]]),
    ([[0, 0], [0, 0], [0, 1]], [[0, 0], [1, 1], [0, 1]]),
    ([[1, 0], [0, 1], [1, 0]], [[0, 0], [0, 0], [1, 1]]),
])
def test_brute_force_tiny_streams_against_literal_transcription(layout):
    hs, fs = layout
    d, w, z = 2, 2, 2
    table = np.zeros((3, d, 2), dtype=np.uint32)
    table[:, :, 0] = hs
    table[:, :, 1] = fs
    idx_of_key = {k: (hs[k], fs[k]) for k in range(3)}
    streams = _tiny_streams(3, 6)
    assert len(streams) > 1000
    for st in streams:
        wantA, wantB = py_literal_seq(d, w, z, idx_of_key, st)
        ids = np.array([k for k, _ in st], np.uint32)
        ops = np.array([o for _, o in st], np.int8)
        h, f, ident = explicit_indices(table, ids)
        for literal in (True, False):
            sk = Sketch(d, w, z)
            sk.seq_apply(h, f, ops, literal=literal)
            assert np.array_equal(sk.A, wantA) and np.array_equal(sk.B, wantB), (st, literal)
        sk = Sketch(d, w, z)
        sk.chunk_apply(h, f, ops, 1, ident)
        assert np.array_equal(sk.A, wantA) and np.array_equal(sk.B, wantB), st


# ---------------------------------------------------------------------------------------
# random streams: theorems, invariants, closed forms
# ---------------------------------------------------------------------------------------

def _turnstile(rng, n, n_keys, del_frac, zipf_a=None):
    """A strict-turnstile stream of key ids (deletes only remove live occurrences)."""
    live = np.zeros(n_keys, np.int64)
    ids, ops = [], []
    for _ in range(n):
        if rng.random() < del_frac and live.sum() > 0:
            k = int(rng.choice(np.flatnonzero(live)))
            live[k] -= 1
            ids.append(k)
            ops.append(-1)
        else:
            k = int(rng.zipf(zipf_a) - 1) % n_keys if zipf_a else int(rng.integers(n_keys))
            live[k] += 1
            ids.append(k)
            ops.append(1)
    return np.array(ids, np.uint32), np.array(ops, np.int8), live


def _key_bytes(ids):
    return np.ascontiguousarray(ids.astype("<u4")).view(np.uint8).reshape(-1, 4)


@pytest.mark.parametrize("seed", range(6))
def test_chunk_size_one_is_sequential(seed):
    rng = np.random.default_rng(seed)
    ids, ops, _ = _turnstile(rng, 3000, 300, 0.3, zipf_a=1.3)
    keys = _key_bytes((ids.astype(np.uint64) * 2654435761) % 2**32)
    a = Sketch(4, 64, 4, 4, seed)
    b = a.copy()
    a.update(keys, ops, S=None)
    b.update(keys, ops, S=1)
    assert np.array_equal(a.A, b.A) and np.array_equal(a.B, b.B)


@pytest.mark.parametrize("seed", range(4))
def test_literal_delete_equals_clamp_delete(seed):
    rng = np.random.default_rng(100 + seed)
    ids, ops, _ = _turnstile(rng, 4000, 500, 0.4, zipf_a=1.2)
    keys = _key_bytes(ids)
    a = Sketch(3, 32, 8, 4, seed)
    b = a.copy()
    a.update(keys, ops, S=None, literal=True)
    b.update(keys, ops, S=None, literal=False)
    assert np.array_equal(a.A, b.A) and np.array_equal(a.B, b.B)


def _bucket_max(sk):
    return sk.B.max(axis=2)


@pytest.mark.parametrize("S", [None, 1, 7, 64, 1000, 5000])
def test_no_underestimation_and_slim_below_bucket_max(S):
    """Appendix II (no under-estimation) and Appendix I (A_i[j] <= max_k B_i[j][k]),
    checked after every chunk of the stream."""
    rng = np.random.default_rng(31)
    ids, ops, _ = _turnstile(rng, 5000, 800, 0.3, zipf_a=1.1)
    keys = _key_bytes(ids)
    sk = Sketch(4, 50, 4, 4, 9)
    step = S or 1
    live = np.zeros(800, np.int64)
    for c0 in range(0, len(ops), step if S else 250):
        c1 = min(len(ops), c0 + (step if S else 250))
        sk.update(keys[c0:c1], ops[c0:c1], S=S)
        np.add.at(live, ids[c0:c1].astype(np.int64), ops[c0:c1].astype(np.int64))
        assert (sk.A <= _bucket_max(sk)).all()
    q = sk.query(_key_bytes(np.arange(800, dtype=np.uint32))).astype(np.int64)
    assert (q >= live).all()


@pytest.mark.parametrize("S", [None, 1, 13, 4096])
def test_fat_is_the_cm_histogram_and_rows_sum_to_the_net_count(S):
    rng = np.random.default_rng(2)
    ids, ops, _ = _turnstile(rng, 6000, 700, 0.25)
    keys = _key_bytes(ids)
    d, w, z = 3, 40, 8
    sk = Sketch(d, w, z, 4, 77)
    sk.update(keys, ops, S=S)
    h, f = sk.index(keys)
    net = int(ops.astype(np.int64).sum())
    for i in range(d):
        hist = np.zeros(w * z, np.int64)
        np.add.at(hist, h[:, i].astype(np.int64) * z + f[:, i], ops.astype(np.int64))
        assert np.array_equal(sk.B[i].reshape(-1).astype(np.int64), hist)
        assert int(sk.B[i].astype(np.int64).sum()) == net


def _collision_free_fat_table(rng, n_keys, d, w, z):
    """Explicit indices where keys share Slim counters but never a Fat counter."""
    table = np.zeros((n_keys, d, 2), np.uint32)
    for i in range(d):
        used = np.zeros(w, np.int64)
        for k in range(n_keys):
            j = int(rng.integers(w))
            while used[j] >= z:
                j = int(rng.integers(w))
            table[k, i] = (j, used[j])
            used[j] += 1
    return table


@pytest.mark.parametrize("S", [None, 1, 2, 5, 31, 100, 10_000])
def test_theorem_slim_counter_is_max_frequency_with_error_free_fat(S):
    """Sec. 3.5 'Derivation of Correct Rate', Theorem 1: with an error-free Fat and insertions
    only, each Slim counter equals the frequency of the most frequent item mapped to it."""
    rng = np.random.default_rng(17)
    n_keys, d, w, z = 60, 3, 8, 16
    table = _collision_free_fat_table(rng, n_keys, d, w, z)
    ids = (rng.zipf(1.3, 3000) - 1) % n_keys
    ids = ids.astype(np.uint32)
    h, f, ident = explicit_indices(table, ids)
    sk = Sketch(d, w, z)
    if S is None:
        sk.seq_apply(h, f, np.ones(len(ids), np.int8))
    else:
        sk.chunk_apply(h, f, np.ones(len(ids), np.int8), S, ident)
    freq = np.bincount(ids, minlength=n_keys)
    want = np.zeros((d, w), np.int64)
    for k in range(n_keys):
        for i in range(d):
            j = table[k, i, 0]
            want[i, j] = max(want[i, j], freq[k])
    assert np.array_equal(sk.A.astype(np.int64), want)


@pytest.mark.parametrize("S", [None, 1, 64, 100_000])
def test_exact_counts_without_collisions(S):
    """No two keys share a Slim counter or a Fat counter (checked): every query is exact,
    with deletions too."""
    rng = np.random.default_rng(23)
    n_keys, d, w, z = 50, 4, 1 << 16, 16
    ids_pool = rng.choice(2**32, n_keys, replace=False).astype(np.uint32)
    sk = Sketch(d, w, z, 4, 1234)
    h, _ = sk.index(_key_bytes(ids_pool))
    for i in range(d):
        assert len(np.unique(h[:, i])) == n_keys, "collision: pick another seed"
    stream, ops, live = _turnstile(rng, 4000, n_keys, 0.3)
    keys = _key_bytes(ids_pool[stream])
    sk.update(keys, ops, S=S)
    q = sk.query(_key_bytes(ids_pool))
    assert np.array_equal(q.astype(np.int64), live)


def _closed_form_chunk(d, w, z, A0, B0, h, f, ops, ident_rows):
    """Order-free form of one CHUNK(S) chunk, derived from its definition: all clamps of a
    counter share the bound M = max_k B1[i][j][k], every raise target T_e <= F_e <= M, so the
    ops of a counter commute and A1 = max(min(A0, M) if the counter saw a delete, max T_e)."""
    B1 = B0.astype(np.int64).copy()
    for t in range(len(ops)):
        for i in range(d):
            B1[i, h[t, i], f[t, i]] += int(ops[t])
    B1 = (B1 % 2**32).astype(np.uint32)
    keys = {}
    for t in range(len(ops)):
        keys.setdefault(bytes(ident_rows[t]), []).append(t)
    A1 = A0.astype(np.int64).copy()
    clamp = np.zeros((d, w), bool)
    for t in range(len(ops)):
        if ops[t] < 0:
            clamp[np.arange(d), h[t]] = True
    M = B1.max(axis=2).astype(np.int64)
    A1 = np.where(clamp, np.minimum(A1, M), A1)
    for ts in keys.values():
        c = sum(1 for t in ts if ops[t] > 0)
        if c == 0:
            continue
        t = ts[0]
        m = min(int(A0[i, h[t, i]]) for i in range(d))
        F = min(int(B1[i, h[t, i], f[t, i]]) for i in range(d))
        T = min(m + c, F)
        for i in range(d):
            A1[i, h[t, i]] = max(A1[i, h[t, i]], T)
    return A1.astype(np.uint32), B1


@pytest.mark.parametrize("seed", range(5))
def test_chunk_equals_its_order_free_closed_form(seed):
    rng = np.random.default_rng(500 + seed)
    d, w, z = 4, 16, 4
    ids, ops, _ = _turnstile(rng, 1500, 120, 0.35, zipf_a=1.4)
    keys = _key_bytes(ids)
    sk = Sketch(d, w, z, 4, seed)
    sk.update(keys[:700], ops[:700], S=None)   # some history
    A0, B0 = sk.A.copy(), sk.B.copy()
    rest_k, rest_o = keys[700:], ops[700:]
    sk.update(rest_k, rest_o, S=len(rest_o))   # one chunk
    h, f = sk.index(rest_k)
    wantA, wantB = _closed_form_chunk(d, w, z, A0, B0, h, f, rest_o, rest_k)
    assert np.array_equal(sk.B, wantB)
    assert np.array_equal(sk.A, wantA)


def test_chunks_restart_at_each_call():
    rng = np.random.default_rng(8)
    ids, ops, _ = _turnstile(rng, 900, 60, 0.2)
    keys = _key_bytes(ids)
    a = Sketch(2, 16, 4, 4, 3)
    b = a.copy()
    a.update(keys, ops, S=300)
    for c0 in range(0, 900, 300):
        b.update(keys[c0:c0 + 300], ops[c0:c0 + 300], S=1000)
    assert np.array_equal(a.A, b.A) and np.array_equal(a.B, b.B)


def test_correct_rate_bound_eq_cr():
    """Sec. 3.5, Eq. (cr): with an error-free Fat and v items of distinct frequencies 1..v,
    the expected fraction of exactly answered items is at least
    (1/v) * sum_l [1 - (1 - (1 - 1/w)^(v-l))^d]."""
    v, d, w, z = 120, 3, 64, 64
    bound = np.mean([1 - (1 - (1 - 1 / w) ** (v - l)) ** d for l in range(1, v + 1)])
    rates = []
    for trial in range(12):
        rng = np.random.default_rng(1000 + trial)
        table = _collision_free_fat_table(rng, v, d, w, z)
        ids = np.repeat(np.arange(v, dtype=np.uint32), np.arange(1, v + 1))
        rng.shuffle(ids)
        h, f, _ = explicit_indices(table, ids)
        sk = Sketch(d, w, z)
        sk.seq_apply(h, f, np.ones(len(ids), np.int8))
        hq, _, _ = explicit_indices(table, np.arange(v, dtype=np.uint32))
        q = sk.query_idx(hq)
        rates.append(float(np.mean(q == np.arange(1, v + 1))))
    assert np.mean(rates) >= bound - 0.02
    # a CM-style Slim (every row incremented) would be far worse: sanity of the margin
    assert bound < 0.99


def test_zero_length_and_edge_shapes():
    sk = Sketch(1, 1, 1, 4, 0)
    sk.update(np.zeros((0, 4), np.uint8), np.zeros(0, np.int8), S=5)
    # three distinct keys on one counter, chunks of 2: chunk 1 raises to min(0+1, 2) = 1,
    # chunk 2 raises to min(1+1, 3) = 2 (SEQ would reach 3: chunking loses accuracy here)
    sk.update(_key_bytes(np.array([1, 2, 3], np.uint32)), np.ones(3, np.int8), S=2)
    assert sk.A.tolist() == [[2]] and sk.B.tolist() == [[[3]]]
    assert sk.query(_key_bytes(np.array([9], np.uint32))).tolist() == [2]
    seq = Sketch(1, 1, 1, 4, 0)
    seq.update(_key_bytes(np.array([1, 2, 3], np.uint32)), np.ones(3, np.int8), S=None)
    assert seq.A.tolist() == [[3]]


def test_chunk_hand_derived_single_counter():
    """CHUNK(S) on one counter (d = w = z = 1), values worked out by hand from the chunk
    definition: the Fat is the plain count, m_e is the chunk-start Slim value, c_e the
    key's inserts in the chunk, T_e = min(m_e + c_e, F_e), clamps use the chunk-end Fat."""
    a, b, c = 1, 2, 3
    sk = Sketch(1, 1, 1, 4, 0)
    steps = [
        # (keys, ops, S, Slim after, Fat after)
        ([a, b, c], [1, 1, 1], 3, 1, 3),    # each key: m=0, c=1, F=3 -> T=1
        ([a, a], [1, 1], 2, 3, 5),          # a: m=1, c=2, F=5 -> T=3
        ([a, b], [1, -1], 2, 4, 5),         # a: m=3, c=1, F=5 -> T=4; clamp min(.,5)
        ([a, a, c], [-1, -1, -1], 3, 2, 2),  # clamp to chunk-end Fat 2
        ([b, b, b], [1, 1, 1], 1, 5, 5),    # S=1: raises 3, 4, 5 one by one
    ]
    for keys, ops, S, want_a, want_b in steps:
        sk.update(_key_bytes(np.array(keys, np.uint32)), np.array(ops, np.int8), S=S)
        assert int(sk.A[0, 0]) == want_a and int(sk.B[0, 0, 0]) == want_b, (keys, ops)


# ---------------------------------------------------------------------------------------
# SF_4 delete rule (Sec. 3.4), the ablation next to SF_F: decrement A_i[h_i(e)] by 1 when it
# is above the bucket sum after the Fat decrement
# ---------------------------------------------------------------------------------------

def _bucket_sum(sk):
    return sk.B.astype(np.uint64).sum(axis=2)


def test_sf4_hand_derived_bucket():
    """d = w = 1, z = 2; e1 lives in slot 0, e2 in slot 1.  Values worked out by hand from the
    Sec. 3.4 rules: ins e1 (A 1), ins e1 (A 2), ins e2 (Bmin 1 <= m 2: no raise), del e1 (bucket
    sum 2, A = 2 is not above it: stays 2; SF_F clamps to the maximum 1), del e1 (sum 1: A 2 -> 1)."""
    h = np.zeros((5, 1), np.uint32)
    f = np.array([[0], [0], [1], [0], [0]], np.uint32)
    ops = np.array([1, 1, 1, -1, -1], np.int8)
    for rule, want in (("sf4", [1, 2, 2, 2, 1]), ("sff", [1, 2, 2, 1, 1])):
        sk = Sketch(1, 1, 2, 4, 0, delete_rule=rule)
        got = []
        for t in range(5):
            sk.seq_apply(h[t:t + 1], f[t:t + 1], ops[t:t + 1])
            got.append(int(sk.A[0, 0]))
        assert got == want, (rule, got)
        assert sk.B[0, 0].tolist() == [0, 1]
    # CHUNK(2) on the same stream: chunks {ins e1, ins e1}, {ins e2, del e1}, {del e1}.
    #   chunk 1: B1 = [2, 0], T(e1) = min(0 + 2, 2) = 2 -> A 2
    #   chunk 2: B1 = [1, 1], T(e2) = min(2 + 1, 1) = 1; delete bound: SF_4 sum 2 (A stays 2),
    #            SF_F max 1 (A -> 1)
    #   chunk 3: B1 = [0, 1], bound 1 for both: A -> 1
    ident = np.array([1, 1, 2, 1, 1], np.uint32).view(np.uint8).reshape(-1, 4)
    for rule, want in (("sf4", [2, 2, 1]), ("sff", [2, 1, 1])):
        sk = Sketch(1, 1, 2, 4, 0, delete_rule=rule)
        got = []
        for c0, c1 in ((0, 2), (2, 4), (4, 5)):
            sk.chunk_apply(h[c0:c1], f[c0:c1], ops[c0:c1], 2, ident[c0:c1])
            got.append(int(sk.A[0, 0]))
        assert got == want, (rule, got)


@pytest.mark.parametrize("S", [None, 1, 64])
def test_sf4_without_deletions_equals_sff(S):
    """SF_4 and SF_F share the insertion rule (Sec. 3.4, 3.5): with no deletion they agree."""
    rng = np.random.default_rng(7)
    ids, ops, _ = _turnstile(rng, 4000, 400, 0.0, zipf_a=1.2)
    keys = _key_bytes(ids)
    a = Sketch(4, 40, 4, 4, 3, delete_rule="sf4")
    b = Sketch(4, 40, 4, 4, 3, delete_rule="sff")
    a.update(keys, ops, S=S)
    b.update(keys, ops, S=S)
    assert np.array_equal(a.A, b.A) and np.array_equal(a.B, b.B)


@pytest.mark.parametrize("seed", range(4))
def test_sf4_chunk_size_one_is_sequential(seed):
    rng = np.random.default_rng(40 + seed)
    ids, ops, _ = _turnstile(rng, 3000, 300, 0.3, zipf_a=1.3)
    keys = _key_bytes(ids)
    a = Sketch(4, 64, 4, 4, seed, delete_rule="sf4")
    b = a.copy()
    a.update(keys, ops, S=None)
    b.update(keys, ops, S=1)
    assert np.array_equal(a.A, b.A) and np.array_equal(a.B, b.B)


@pytest.mark.parametrize("S", [None, 1, 7, 256])
def test_sf4_slim_below_bucket_sum_and_no_underestimation(S):
    """Sec. 3.4 states that a Slim counter never exceeds the sum of its Fat bucket; the SF_F
    no-under-estimation proof (Appendix II) carries over with the bucket sum in place of the
    bucket maximum (sum >= max >= every item's Fat counter).  Checked after every chunk."""
    rng = np.random.default_rng(55)
    ids, ops, _ = _turnstile(rng, 4000, 600, 0.35, zipf_a=1.1)
    keys = _key_bytes(ids)
    sk = Sketch(3, 30, 4, 4, 11, delete_rule="sf4")
    step = S or 1
    live = np.zeros(600, np.int64)
    for c0 in range(0, len(ops), step if S else 1):
        c1 = min(len(ops), c0 + step)
        sk.update(keys[c0:c1], ops[c0:c1], S=S)
        np.add.at(live, ids[c0:c1].astype(np.int64), ops[c0:c1].astype(np.int64))
        assert (sk.A.astype(np.uint64) <= _bucket_sum(sk)).all()
    q = sk.query(_key_bytes(np.arange(600, dtype=np.uint32))).astype(np.int64)
    assert (q >= live).all()


@pytest.mark.parametrize("S", [None, 1, 13, 500])
def test_sf4_decrement_is_a_clamp_to_the_bucket_sum(S):
    """Because A <= bucket sum holds before every deletion (Sec. 3.4), "decrement by 1 when
    above the sum after the Fat decrement" lowers A exactly to that sum: the SF_4 deletion is
    the SF_F clamp with the bucket sum in place of the bucket maximum.  Checked after each
    chunk: every Slim counter that went down equals its bucket sum, and only counters that a
    deletion in the chunk hashed to went down."""
    rng = np.random.default_rng(77)
    ids, ops, _ = _turnstile(rng, 3000, 300, 0.4, zipf_a=1.3)
    keys = _key_bytes(ids)
    sk = Sketch(2, 16, 3, 4, 5, delete_rule="sf4")
    h, _ = sk.index(keys)
    step = S or 1
    for c0 in range(0, len(ops), step):
        c1 = min(len(ops), c0 + step)
        before = sk.A.copy()
        sk.update(keys[c0:c1], ops[c0:c1], S=S)
        lowered = sk.A < before
        assert (sk.A[lowered].astype(np.uint64) == _bucket_sum(sk)[lowered]).all()
        # a counter can only go down through a deletion of a key hashed to it in this chunk
        touched = np.zeros_like(lowered)
        for t in range(c0, c1):
            if ops[t] < 0:
                touched[np.arange(sk.d), h[t]] = True
        assert not (lowered & ~touched).any()
