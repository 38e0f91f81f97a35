"""The seeded input generators keep the recipe the measurements state: Zipf(s) frequencies,
distinct ids and flows, deletions drawn only from inserted occurrences, and strict-turnstile
order in the interleaved streams (CPU, small sizes)."""
import numpy as np
import pytest
import torch

import workloads as wl


def _rows(t):
    """Rows of a (n, k) uint8 tensor as hashable bytes."""
    a = t.numpy()
    return [bytes(r) for r in a]


@pytest.mark.parametrize("s", [0.0, 1.0, 3.0])
def test_zipf_ranks_follow_the_pmf(s):
    n, m = 50, 400_000
    g = wl._gen(11, "cpu")
    r = wl.sample_ranks(m, n, s, g).numpy()
    assert r.min() >= 0 and r.max() < n
    k = np.arange(1, n + 1, dtype=np.float64)
    p = k ** -s / np.sum(k ** -s)
    obs = np.bincount(r, minlength=n)
    exp = p * m
    keep = exp >= 5                      # chi-square over the cells with enough expected mass
    chi2 = float(np.sum((obs[keep] - exp[keep]) ** 2 / exp[keep]))
    dof = int(keep.sum()) - 1
    assert chi2 < dof + 6.0 * np.sqrt(2.0 * dof) + 10.0, (s, chi2, dof)
    if s == 3.0:                          # the hottest rank holds 1 / H_{50,3} ~ 83 % of the draws
        assert abs(obs[0] / m - p[0]) < 0.005 and p[0] > 0.83


def test_distinct_ids_and_flows():
    g = wl._gen(5, "cpu")
    ids = wl.distinct_ids(20_000, 64, g)
    assert torch.unique(ids).numel() == 20_000
    fl = wl.distinct_5tuples(20_000, g)
    assert fl.shape == (20_000, 13) and len(set(_rows(fl))) == 20_000
    assert set(fl[:, 12].tolist()) <= {1, 6, 17}   # protocol byte: ICMP, TCP, UDP


def test_flow_deletes_remove_inserted_occurrences():
    ins, dels, flows = wl.flows_with_deletes(60_000, 5_000, 1.0, 0.1, seed=3)
    assert dels.shape[0] == 6_000
    fl = set(_rows(flows))
    ins_rows, del_rows = _rows(ins), _rows(dels)
    assert set(ins_rows) <= fl
    from collections import Counter
    ci, cd = Counter(ins_rows), Counter(del_rows)
    assert all(cd[k] <= ci[k] for k in cd)           # a delete never exceeds the insertions of its key


@pytest.mark.parametrize("key_bytes", [4, 8])
def test_mixed_stream_is_strict_turnstile(key_bytes):
    st, table = wl.mixed_stream(50_000, 3_000, 1.2, 0.2, key_bytes, seed=9)
    keys, ops = st.keys, st.ops.numpy().astype(np.int64)
    assert keys.shape == (50_000, key_bytes) and set(np.unique(ops).tolist()) == {-1, 1}
    assert abs(float((ops < 0).mean()) - 0.2) < 1e-3
    assert set(_rows(keys)) <= set(_rows(table))
    kid = np.frombuffer(keys.numpy().tobytes(), dtype=np.uint32 if key_bytes == 4 else np.uint64)
    order = np.argsort(kid, kind="stable")           # per key, in stream order
    sk, so = kid[order], ops[order]
    starts = np.r_[True, sk[1:] != sk[:-1]]
    run = np.cumsum(so)
    base = np.maximum.accumulate(np.where(starts, np.arange(len(sk)), 0))
    before = np.where(base > 0, run[base - 1], 0)
    assert (run - before).min() >= 0                 # no key's net count ever goes negative


def test_same_seed_same_stream():
    a = wl.mixed_stream(5_000, 700, 1.0, 0.1, 4, seed=21)[0]
    b = wl.mixed_stream(5_000, 700, 1.0, 0.1, 4, seed=21)[0]
    c = wl.mixed_stream(5_000, 700, 1.0, 0.1, 4, seed=22)[0]
    assert torch.equal(a.keys, b.keys) and torch.equal(a.ops, b.ops)
    assert not torch.equal(a.keys, c.keys)
