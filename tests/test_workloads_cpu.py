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


def test_zipf_table_is_built_on_the_host():
    """The Zipf table of a device stream equals the host table bit for bit (a device scan may
    change the order of its partial sums between runs)."""
    c = wl.zipf_cdf(1 << 16, 1.2, "cpu")
    assert c.dtype == torch.float64 and float(c[-1]) == 1.0
    assert bool((c[1:] >= c[:-1]).all())
    k = torch.arange(1, (1 << 16) + 1, dtype=torch.float64)
    assert torch.equal(c, torch.cumsum(k ** -1.2, 0) / torch.cumsum(k ** -1.2, 0)[-1])


@pytest.mark.gpu
def test_device_streams_repeat_for_a_seed():
    """Two calls with one seed give the same device stream, at the size of the out-of-L2
    workload's id table (2^26 ranks, many scan tiles)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    a, ta = wl.mixed_stream(1 << 22, 1 << 26, 1.2, 0.2, 8, seed=5, device=dev)
    b, tb = wl.mixed_stream(1 << 22, 1 << 26, 1.2, 0.2, 8, seed=5, device=dev)
    assert torch.equal(ta, tb)
    assert torch.equal(a.keys, b.keys) and torch.equal(a.ops, b.ops)
    g1, g2 = wl._gen(9, dev), wl._gen(9, dev)
    assert torch.equal(wl.sample_ranks(1 << 20, 1 << 26, 0.99, g1, dev),
                       wl.sample_ranks(1 << 20, 1 << 26, 0.99, g2, dev))
