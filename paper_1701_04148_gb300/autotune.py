"""Autotuner for the batched many-sketch update.

What it tunes, in three stages on the real batch:
1. The round count R. Every sketch k gets the chunk size `S_k = ceil(N_k / R)` (at least 2, at most
   SF_MAX_CHUNK), so every stream spreads over about R rounds of one launch. Chunk size is part of the
   semantics: it is recorded in the plan and in each sketch's parameters, and the CPU oracle takes it
   as an input. The largest R (smallest chunks, closest to one-at-a-time semantics) whose throughput
   is within `tolerance` of the best candidate is kept.  Candidates run from 2 to 1024.  Throughput
   grows with the chunk size (fewer rounds, fewer grid barriers) until the dictionaries of a launch
   no longer fit L2 beside the counters.  A candidate whose sketches would need more device memory
   than `mem_budget` is skipped: each chunk slot reserves dictionary entries, in the sketch's scratch,
   or -- with SF_FLAG_SHARED_DICT sketches and `dict_arena_bytes` -- in one arena that the batch's
   launch groups reuse one after another.  The plan records whether the fastest tried R lay inside
   the range or at its end.
2. The launch shape at that R: threads per block (512, 256 or 128, with 512 / threads blocks per SM,
   so every shape runs the same number of threads). The fastest shape is kept; shapes are not
   semantic.
3. The launch-group budget at that R and shape: the default (3/4 of L2), half of L2, or one launch
   for every sketch. The fastest is kept; grouping is not semantic either.

How it times: one warm-up call, then `trials` calls per candidate, sketches re-initialised between
calls. The plan is cached as JSON, keyed by a hash of the batch shape.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

SF_MAX_CHUNK = 1 << 20
ROUND_CANDIDATES = (2, 4, 8, 16, 32, 64, 256, 1024)
BLOCK_CANDIDATES = (512, 256, 128)


def chunk_sizes(ns, rounds: int, s_min: int = 2, s_max: int = SF_MAX_CHUNK):
    return [min(s_max, max(s_min, -(-int(n) // rounds))) for n in ns]


def choose_rounds(results: dict, tolerance: float) -> int:
    """The largest round count (smallest chunks, closest to one-at-a-time semantics) whose
    throughput is within `tolerance` of the best candidate's."""
    top = max(results.values())
    return max(R for R, v in results.items() if v >= (1.0 - tolerance) * top)


def choose_fastest(results: dict, order):
    """The fastest candidate of a non-semantic choice; on a tie the one listed first in `order`."""
    top = max(results.values())
    return next(c for c in order if c in results and results[c] == top)


def bracketed(results: dict) -> bool:
    """True when the fastest round count is not at either end of the candidates tried."""
    best = max(results, key=lambda R: results[R])
    return min(results) < best < max(results)


def shape_key(widths, ns, d: int, z: int, key_bytes: int) -> str:
    h = hashlib.sha256()
    h.update(json.dumps([list(map(int, widths)), list(map(int, ns)), d, z, key_bytes]).encode())
    return h.hexdigest()[:24]


def _time_batch(sf, torch, sks, streams, graph, slots, trials, block=None, group=None, arena=None):
    b = sf.Batch(len(sks), graph=graph, max_round_slots=slots, block_threads=block, group_bytes=group,
                 dict_arena_bytes=arena)
    items = [(sk, k, o) for sk, (k, o) in zip(sks, streams)]
    for sk in sks:
        sk.reset()
    b.update(items)
    b.sync()
    best = float("inf")
    for _ in range(trials):
        for sk in sks:
            sk.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.update(items)
        b.sync()
        best = min(best, time.perf_counter() - t0)
    b.close()
    return best


def sketch_bytes(widths, chunks, d: int, z: int, shared_dict: bool = False) -> int:
    """Device bytes of the batch's sketches (Fat, Slim and scratch of sf_required_bytes: with
    shared_dict, SF_FLAG_SHARED_DICT sketches, whose dictionaries come from the batch's arena)."""
    import paper_1701_04148_gb300 as sf
    total = 0
    flags = sf.SF_FLAG_SHARED_DICT if shared_dict else 0
    for w, c in zip(widths, chunks):
        fb, sb, xb = sf.required_bytes(sf.make_params(d, int(w), z, 4, 0, int(c), flags))
        total += fb + sb + xb
    return total


def _read_cache(path: str) -> dict:
    """The plan cache, or {} when it is missing or unreadable (then the batch is tuned again)."""
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def tune(make_sketches, streams, ns, candidates=ROUND_CANDIDATES, blocks=BLOCK_CANDIDATES, group_budgets=None,
         tolerance: float = 0.05, trials: int = 1, graph: bool = True, cache_path: str | None = None,
         cache_key: str | None = None, log=None, widths=None, d: int = 4, z: int = 16, mem_budget: int | None = None,
         dict_arena_bytes: int | None = None):
    """make_sketches(chunks) -> list of Sketch; streams: list of (keys, ops) device tensors.
    dict_arena_bytes: make_sketches creates SF_FLAG_SHARED_DICT sketches, and every timed batch gets
    a dictionary arena of this size (the memory check then counts the sketches without
    dictionaries, plus the arena).
    group_budgets: launch-group budgets to try (None entries: the library default); by default the
    default, half of L2 and 0 (one launch).  widths (with d, z): the sketches' widths, to skip round
    counts whose sketches exceed mem_budget bytes (default: a sixth of the device's memory, so that a
    caller can hold a second set of the tuned sketches beside its inputs, and the choice does not
    depend on what else happens to be allocated).
    Returns {"rounds", "chunks", "block_threads", "group_bytes", "graph", "trials", ...}."""
    import torch

    import paper_1701_04148_gb300 as sf

    if cache_path and cache_key:
        cache = _read_cache(cache_path)
        if cache_key in cache:
            return cache[cache_key]
    if group_budgets is None:
        l2 = torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size
        group_budgets = (None, l2 // 2, 0)
    total = sum(int(n) for n in ns)
    say = log or (lambda m: None)
    if mem_budget is None:
        mem_budget = torch.cuda.get_device_properties(torch.cuda.current_device()).total_memory // 6
    skipped = []

    # stage 1: round count at the default shape and grouping
    by_rounds = {}
    for R in candidates:
        chunks = chunk_sizes(ns, R)
        need = (sketch_bytes(widths, chunks, d, z, dict_arena_bytes is not None) + (dict_arena_bytes or 0)
                if widths is not None else 0)
        if widths is not None and need > mem_budget:
            skipped.append(R)
            say(f"autotune: R={R} skipped (sketches above the memory budget)")
            continue
        slots = sum((c + 31) // 32 * 32 for c in chunks)
        sks = make_sketches(chunks)
        by_rounds[R] = total / _time_batch(sf, torch, sks, streams, graph, slots, trials, arena=dict_arena_bytes)
        say(f"autotune: R={R} -> {by_rounds[R] / 1e9:.3f} G updates/s")
        for sk in sks:
            sk.close()
        del sks
    chosen = choose_rounds(by_rounds, tolerance)
    chunks = chunk_sizes(ns, chosen)
    slots = sum((c + 31) // 32 * 32 for c in chunks)
    sks = make_sketches(chunks)
    # stage 2: launch shape at that round count
    by_block = {}
    for blk in blocks:
        by_block[blk] = total / _time_batch(sf, torch, sks, streams, graph, slots, trials, block=blk,
                                            arena=dict_arena_bytes)
        say(f"autotune: R={chosen} block={blk} -> {by_block[blk] / 1e9:.3f} G updates/s")
    block = choose_fastest(by_block, blocks)
    # stage 3: launch-group budget at that round count and shape
    by_group = {}
    for gbytes in group_budgets:
        by_group[gbytes] = total / _time_batch(sf, torch, sks, streams, graph, slots, trials, block=block,
                                               group=gbytes, arena=dict_arena_bytes)
        say(f"autotune: R={chosen} block={block} group={gbytes} -> {by_group[gbytes] / 1e9:.3f} G updates/s")
    group = choose_fastest(by_group, list(group_budgets))
    for sk in sks:
        sk.close()
    del sks
    plan = {"rounds": chosen, "chunks": chunks, "graph": graph, "round_slots": slots,
            "block_threads": block, "group_bytes": group,
            "trials": {str(k): v for k, v in by_rounds.items()},
            "trials_block": {str(k): v for k, v in by_block.items()},
            "trials_group": {("default" if k is None else str(k)): v for k, v in by_group.items()},
            "best_rounds_bracketed": bracketed(by_rounds), "rounds_skipped_for_memory": skipped,
            "mem_budget": mem_budget, "tolerance": tolerance, "dict_arena_bytes": dict_arena_bytes}
    if cache_path and cache_key:
        cache = _read_cache(cache_path)
        cache[cache_key] = plan
        os.makedirs(os.path.dirname(cache_path) or ".", exist_ok=True)
        # several processes (one per GPU) may tune at once: write a private file, then rename it
        # over the cache, so a reader sees the old or the new file, never half of one
        tmp = f"{cache_path}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f)
        os.replace(tmp, cache_path)
    return plan
