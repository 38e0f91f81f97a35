"""Seeded synthetic workloads for the SF-sketch hot path.

This module only draws random inputs (keys, +1/-1 operations, query sets).  It holds none
of the sketch's arithmetic, so both the CUDA path and the CPU oracle may consume what it
makes.  Everything is a torch tensor on the requested device; the same seed on the same
device type gives the same stream (every step is deterministic there: seeded draws, sorts,
gathers; the one floating-point reduction, the Zipf table, runs on the host).

Recipe (stand-ins for the paper's YCSB uniform/Zipf-0.99 traces and campus trace, Sec. 5.1,
which are not available):
  * Zipf(s) over a finite support of n ranks: P(rank k) proportional to k^-s, k = 1..n
    (s = 0 is uniform), sampled by inverse CDF: a float64 cumulative table and a binary
    search (``torch.searchsorted``) of uniform float64 draws.
  * ranks map to key ids through a seeded random permutation, so hot keys are not small
    integers.
  * distinct ids: uniform random 32/64-bit values with duplicates removed, or 13-byte
    5-tuples {u32 src, u32 dst, u16 sport, u16 dport, u8 proto} packed little-endian.
  * strict-turnstile deletions: every delete removes an occurrence inserted earlier.
"""
from __future__ import annotations

import dataclasses
import math

import torch

ZIPF_SWEEP = (0.0, 0.5, 1.0, 1.5, 2.0, 3.0)


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFF_FFFF_FFFF_FFFF)
    return g


def zipf_cdf(n: int, s: float, device="cpu") -> torch.Tensor:
    """float64 cumulative Zipf(s) table over ranks 1..n, built on the host and then moved to
    `device`: a scan on the GPU may add its partial sums in a different order from run to run,
    which moves the table's last bits and, with them, some sampled ranks."""
    k = torch.arange(1, n + 1, dtype=torch.float64)
    p = torch.pow(k, -float(s))
    c = torch.cumsum(p, 0)
    return (c / c[-1]).to(device)


def sample_ranks(n_samples: int, n: int, s: float, g: torch.Generator, device="cpu",
                 block: int = 1 << 26) -> torch.Tensor:
    """int64 Zipf(s) ranks in [0, n) (rank 0 is the most frequent)."""
    cdf = zipf_cdf(n, s, device)
    out = torch.empty(n_samples, dtype=torch.int64, device=device)
    for b0 in range(0, n_samples, block):
        b1 = min(n_samples, b0 + block)
        u = torch.rand(b1 - b0, dtype=torch.float64, generator=g, device=device)
        r = torch.searchsorted(cdf, u, right=True)
        out[b0:b1] = torch.clamp(r, max=n - 1)
    return out


def distinct_ids(n: int, bits: int, g: torch.Generator, device="cpu") -> torch.Tensor:
    """n distinct uniform random ids of `bits` bits (int64 holding the bit pattern), in random order."""
    have = torch.empty(0, dtype=torch.int64, device=device)
    while have.numel() < n:
        m = int((n - have.numel()) * 1.05) + 16
        if bits == 32:
            x = torch.randint(0, 1 << 32, (m,), dtype=torch.int64, generator=g, device=device)
        else:
            hi = torch.randint(0, 1 << 32, (m,), dtype=torch.int64, generator=g, device=device)
            lo = torch.randint(0, 1 << 32, (m,), dtype=torch.int64, generator=g, device=device)
            x = (hi << 32) | lo
        have = torch.unique(torch.cat([have, x]))
    perm = torch.randperm(have.numel(), generator=g, device=device)[:n]
    return have[perm]


def ids_to_bytes(ids: torch.Tensor, key_bytes: int) -> torch.Tensor:
    """Packed little-endian key bytes (n, key_bytes) uint8 of int64 ids."""
    n = ids.numel()
    shifts = torch.arange(0, 8 * key_bytes, 8, device=ids.device, dtype=torch.int64)
    b = (ids.reshape(n, 1) >> shifts.reshape(1, -1)) & 0xFF
    return b.to(torch.uint8).contiguous()


def distinct_5tuples(n: int, g: torch.Generator, device="cpu") -> torch.Tensor:
    """n distinct 13-byte flow keys {u32 src, u32 dst, u16 sport, u16 dport, u8 proto}."""
    have = torch.empty((0, 13), dtype=torch.uint8, device=device)
    while have.shape[0] < n:
        m = int((n - have.shape[0]) * 1.02) + 16
        raw = torch.randint(0, 256, (m, 13), dtype=torch.uint8, generator=g, device=device)
        # bias the protocol byte toward TCP/UDP/ICMP like real traffic
        proto = torch.tensor([6, 17, 1, 6], dtype=torch.uint8, device=device)
        raw[:, 12] = proto[torch.randint(0, 4, (m,), generator=g, device=device)]
        have = torch.unique(torch.cat([have, raw]), dim=0)
    perm = torch.randperm(have.shape[0], generator=g, device=device)[:n]
    return have[perm].contiguous()


def gather_keys(id_table: torch.Tensor, ranks: torch.Tensor) -> torch.Tensor:
    return id_table.index_select(0, ranks).contiguous()


def turnstile_interleave(n_total: int, del_frac: float, g: torch.Generator, device="cpu"):
    """Order of a mixed stream where deletes remove earlier inserts.

    Returns (ins_index, is_delete): position p of the stream is an operation on insert
    occurrence ins_index[p] (an insert when is_delete[p] is False, the delete of that
    earlier insert otherwise).  About del_frac of the stream are deletes; each delete is
    placed uniformly at random after its insert."""
    n_ins = int(round(n_total * (1.0 - del_frac)))
    n_del = n_total - n_ins
    victims = torch.randperm(n_ins, generator=g, device=device)[:n_del]
    pos_ins = torch.arange(n_ins, dtype=torch.float64, device=device)
    u = torch.rand(n_del, dtype=torch.float64, generator=g, device=device)
    vf = victims.to(torch.float64)
    pos_del = vf + 0.5 + u * (n_ins - vf - 0.5)  # strictly after its insert
    pos = torch.cat([pos_ins, pos_del])
    order = torch.argsort(pos, stable=True)
    idx = torch.cat([torch.arange(n_ins, device=device), victims])[order]
    is_del = (order >= n_ins)
    return idx, is_del


@dataclasses.dataclass
class Stream:
    """One call's worth of updates (keys packed (n, key_bytes) uint8, ops int8 +1/-1)."""
    keys: torch.Tensor
    ops: torch.Tensor


# --------------------------------------------------------------------------------------
# Workloads shaped like the configurations this library is measured on.
# --------------------------------------------------------------------------------------

def insert_only_u32(n_updates: int, n_distinct: int, s: float, seed: int, device="cpu"):
    """Insertion-only u32 stream: Zipf(s) over n_distinct random u32 ids.
    Returns (keys (n,4) uint8, distinct ids (n_distinct,4) uint8)."""
    g = _gen(seed, device)
    ids = distinct_ids(n_distinct, 32, g, device)
    ranks = sample_ranks(n_updates, n_distinct, s, g, device)
    table = ids_to_bytes(ids, 4)
    return gather_keys(table, ranks), table


def flows_with_deletes(n_inserts: int, n_flows: int, s: float, del_frac: float, seed: int,
                       device="cpu"):
    """5-tuple workload: n_inserts Zipf(s) draws over n_flows distinct 13-byte flows, then
    deletes of a random del_frac of the inserted occurrences, in random order.
    Returns (insert keys (n,13), delete keys (m,13), flows (n_flows,13))."""
    g = _gen(seed, device)
    flows = distinct_5tuples(n_flows, g, device)
    ranks = sample_ranks(n_inserts, n_flows, s, g, device)
    ins = gather_keys(flows, ranks)
    n_del = int(round(n_inserts * del_frac))
    victims = torch.randperm(n_inserts, generator=g, device=device)[:n_del]
    dels = ins.index_select(0, victims).contiguous()
    return ins, dels, flows


def mixed_stream(n_total: int, n_distinct: int, s: float, del_frac: float, key_bytes: int,
                 seed: int, device="cpu"):
    """Interleaved strict-turnstile stream of u32/u64 keys.
    Returns (Stream, distinct id bytes (n_distinct, key_bytes))."""
    g = _gen(seed, device)
    ids = distinct_ids(n_distinct, 8 * key_bytes, g, device)
    table = ids_to_bytes(ids, key_bytes)
    idx, is_del = turnstile_interleave(n_total, del_frac, g, device)
    n_ins = int(round(n_total * (1.0 - del_frac)))
    ranks = sample_ranks(n_ins, n_distinct, s, g, device)
    keys = table.index_select(0, ranks.index_select(0, idx)).contiguous()
    ops = torch.where(is_del, torch.tensor(-1, dtype=torch.int8, device=device),
                      torch.tensor(1, dtype=torch.int8, device=device)).contiguous()
    return Stream(keys, ops), table


def many_sketch_plan(n_sketches: int, seed: int, w_log2=(10.0, 16.0), n_log10=(4.0, 7.0),
                     s_range=(0.5, 1.5), scale: float = 1.0):
    """Shapes of a many-node batch: per sketch Slim width w_k = round(2^U(a,b)),
    stream length N_k = round(10^U(c,d) * scale), Zipf s_k ~ U(s_lo, s_hi),
    distinct ids 10 * w_k.  Returns a list of dicts (CPU-side, small)."""
    g = _gen(seed, "cpu")
    u = torch.rand(n_sketches, 3, dtype=torch.float64, generator=g)
    out = []
    for k in range(n_sketches):
        w = int(round(2.0 ** (w_log2[0] + (w_log2[1] - w_log2[0]) * float(u[k, 0]))))
        n = max(1, int(round((10.0 ** (n_log10[0] + (n_log10[1] - n_log10[0]) * float(u[k, 1]))) * scale)))
        s = s_range[0] + (s_range[1] - s_range[0]) * float(u[k, 2])
        out.append({"w": w, "n": n, "s": s, "distinct": 10 * w, "seed": seed * 100003 + k})
    return out


def query_mix(present: torch.Tensor, n: int, hot_frac: float, s: float, seed: int,
              device="cpu", key_bits: int = 32):
    """n query keys: hot_frac drawn Zipf(s) from `present` (rows of packed id bytes),
    the rest uniform random ids of key_bits bits (absent with overwhelming probability)."""
    g = _gen(seed, device)
    n_hot = int(round(n * hot_frac))
    kb = present.shape[1]
    ranks = sample_ranks(n_hot, present.shape[0], s, g, device)
    hot = present.index_select(0, ranks)
    cold = ids_to_bytes(distinct_ids(n - n_hot, key_bits, g, device), kb) if n > n_hot else \
        torch.empty((0, kb), dtype=torch.uint8, device=device)
    q = torch.cat([hot, cold])
    return q[torch.randperm(n, generator=g, device=device)].contiguous()


def log_uniform_int(lo_log2: float, hi_log2: float, g: torch.Generator) -> int:
    u = float(torch.rand(1, dtype=torch.float64, generator=g))
    return int(round(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)))


def poisson_gaps(n: int, rate_per_s: float, g: torch.Generator) -> torch.Tensor:
    """Exponential inter-arrival gaps (seconds) of a Poisson process."""
    u = torch.rand(n, dtype=torch.float64, generator=g)
    return -torch.log1p(-u) / rate_per_s


def expected_log_uniform(lo_log2: float, hi_log2: float) -> float:
    a, b = lo_log2 * math.log(2), hi_log2 * math.log(2)
    return (math.exp(b) - math.exp(a)) / (b - a)
