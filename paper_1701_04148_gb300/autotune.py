"""Autotuner for the batched many-sketch update.

What it tunes:
- The round count R of a batch. Every sketch k gets the chunk size `S_k = ceil(N_k / R)`
  (at least 2, at most SF_MAX_CHUNK), so every stream spreads over about R rounds of one launch.
- Whether the launch is replayed from a CUDA graph.

Chunk size is part of the semantics: it is recorded in the plan and in each sketch's
parameters, and the CPU oracle takes it as an input. The block shape is fixed by the kernel's
register budget (512 threads, one block per SM); the tile is a warp-iteration of 32 updates.

How it chooses:
- It times each candidate on the real batch: one warm-up call, then `trials` calls. Sketches
  are re-initialised between calls.
- It keeps the largest R (smallest chunks, closest to one-at-a-time semantics) whose throughput
  is within `tolerance` of the best candidate.
- The plan is cached as JSON, keyed by a hash of the batch shape.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

SF_MAX_CHUNK = 1 << 20


def chunk_sizes(ns, rounds: int, s_min: int = 2, s_max: int = SF_MAX_CHUNK):
    return [min(s_max, max(s_min, -(-int(n) // rounds))) for n in ns]


def choose_rounds(results: dict, tolerance: float) -> int:
    """The largest round count (smallest chunks, closest to one-at-a-time semantics) whose
    throughput is within `tolerance` of the best candidate's."""
    top = max(results.values())
    return max(R for R, v in results.items() if v >= (1.0 - tolerance) * top)


def shape_key(widths, ns, d: int, z: int, key_bytes: int) -> str:
    h = hashlib.sha256()
    h.update(json.dumps([list(map(int, widths)), list(map(int, ns)), d, z, key_bytes]).encode())
    return h.hexdigest()[:24]


def tune(make_sketches, streams, ns, candidates=(16, 64, 256, 1024), tolerance: float = 0.05, trials: int = 1,
         graph: bool = True, cache_path: str | None = None, cache_key: str | None = None, log=None):
    """make_sketches(chunks) -> list of Sketch; streams: list of (keys, ops) device tensors.
    Returns {"rounds": R, "chunks": [S_k], "graph": bool, "trials": {R: updates/s}}."""
    import torch

    import paper_1701_04148_gb300 as sf

    if cache_path and cache_key and os.path.exists(cache_path):
        cache = json.load(open(cache_path))
        if cache_key in cache:
            return cache[cache_key]
    total = sum(int(n) for n in ns)
    results = {}
    for R in candidates:
        chunks = chunk_sizes(ns, R)
        slots = sum((c + 31) // 32 * 32 for c in chunks)
        sks = make_sketches(chunks)
        b = sf.Batch(len(sks), graph=graph, max_round_slots=slots)
        items = [(sk, k, o) for sk, (k, o) in zip(sks, streams)]
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
        results[R] = total / best
        if log:
            log(f"autotune: R={R} -> {results[R] / 1e9:.3f} G updates/s")
        b.close()
        for sk in sks:
            sk.close()
        del sks
    chosen = choose_rounds(results, tolerance)
    chunks = chunk_sizes(ns, chosen)
    plan = {"rounds": chosen, "chunks": chunks, "graph": graph,
            "round_slots": sum((c + 31) // 32 * 32 for c in chunks),
            "trials": {str(k): v for k, v in results.items()}, "tolerance": tolerance}
    if cache_path and cache_key:
        cache = json.load(open(cache_path)) if os.path.exists(cache_path) else {}
        cache[cache_key] = plan
        os.makedirs(os.path.dirname(cache_path) or ".", exist_ok=True)
        json.dump(cache, open(cache_path, "w"))
    return plan
