#!/usr/bin/env python3
"""Benchmark of the SF-sketch hot path on GB300: one JSON line on rank 0.

Workload (one step = one pass of the whole path over one batch of synthetic input): for each
Zipf exponent s in {0, 0.5, 1, 1.5, 2, 3}, a fresh sketch (d=4, w=2^18, z=16, 13-byte 5-tuple
keys, chunk 65,536) takes 32,000,000 inserts drawn Zipf(s) over 1,000,000 distinct flows, then
deletes of a random 10 % of the inserted occurrences; its Slim-subsketch is exported and all
1,000,000 flows are queried.  value = (inserts + deletes + queries) of all ranks / step time.

The default run (--workload all) embeds the other measured configurations in the same line:
"batched" (1,024 uneven sketches in one graph launch vs one call per sketch), "out_of_l2"
(10^9 u64 keys on a 1 GiB Fat), "one_at_a_time" (the paper's rule, chunk 1) and "serving" (the
collector loop, p50/p99).  Each can also be run alone with --workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (plain sequential C, one core) on a bounded sample of the
same workload.  Under torchrun (N > 1) every rank runs an independent replica (its own seeds);
only timing is reduced across ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "M inserts/s + M queries/s, bit-exact; batched vs plain speedup; p99 query ms"
SWEEP = (0.0, 0.5, 1.0, 1.5, 2.0, 3.0)
D, W, Z, KB, S = 4, 1 << 18, 16, 13, 65536
N_INS, N_FLOWS, DEL_FRAC = 32_000_000, 1_000_000, 0.10
SEED0 = 2
# repetitions of each end-to-end form (interleaved); each form reports its median, which stays
# put when up to two repetitions run slow.  When a form's repetitions differ by more than
# E2E_SPREAD, E2E_EXTRA more rounds of all forms run and the median is taken over all of them.
E2E_REPETITIONS = 5
E2E_EXTRA = 4
E2E_SPREAD = 1.15
L2_OPS_PER_UPDATE = 4 * D   # d Fat RMW + d Fat reads + d Slim reads + d Slim RMW (Sec. 3.4/3.5 rules)
L2_OPS_PER_QUERY = D        # d Slim gathers (Sec. 3.1 query)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def seed_for(rank, idx):
    return SEED0 + 1000 * rank + idx


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="sf_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu_index)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index_for(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids) and ids[local_rank].isdigit():
            return int(ids[local_rank])
    return local_rank


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def l2_random_peaks(L, dev, stream):
    """Best of three rates (G ops/s) of sf_bench_random_access on a 64 MiB buffer: 32-bit loads
    (kind 2), RED.ADD (kind 0) and the 1:1 reduce/load mix (kind 5)."""
    import torch
    buf = torch.zeros(1 << 24, dtype=torch.int32, device=dev)
    h_st = int(stream.cuda_stream)
    out = {}
    for name, kind in (("ld", 2), ("red", 0), ("mix", 5)):
        L.sf_bench_random_access(buf.data_ptr(), buf.numel(), 1 << 28, kind, 0, h_st)
        best = 0.0
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            L.sf_bench_random_access(buf.data_ptr(), buf.numel(), 1 << 28, kind, 0, h_st)
            b.record(stream)
            torch.cuda.synchronize()
            best = max(best, (1 << 28) / a.elapsed_time(b) / 1e6)
        out[name] = best
    del buf
    return out


CHUNK_KERNEL_SOURCES = ("sf_update_kernels.cuh", "sf_update.cu", "sf_device.cuh", "sf_internal.h")


def code_without_comments(text: str) -> str:
    """C/C++/CUDA source with its comments removed and every run of whitespace made one space;
    string and character literals (the kernels' inline PTX) are kept as they are."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def chunk_kernel_source_sha256():
    """sha256 over the code (comments and layout aside) of the files the chunk kernels are compiled
    from, in CHUNK_KERNEL_SOURCES order: a traffic record stays valid across comment edits."""
    h = hashlib.sha256()
    for name in CHUNK_KERNEL_SOURCES:
        text = open(os.path.join(ROOT, "paper_1701_04148_gb300", "csrc", name), encoding="utf-8").read()
        h.update(code_without_comments(text).encode())
        h.update(b"\0")
    return h.hexdigest()


def traffic_record(name="chunk_single_kernel_traffic.json"):
    """DRAM bytes per update of a chunk kernel from a committed ncu summary (the single-iteration
    kernel's by default; chunk_update_kernel_traffic.json for the multi-iteration kernel), if the
    kernel sources have not changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    rec = json.load(open(p))
    return rec if rec.get("kernel_source_sha256") == chunk_kernel_source_sha256() else None


# ------------------------------------------------------------------------------------------
# reference arm: the CPU oracle on a bounded sample of the same workload
# ------------------------------------------------------------------------------------------

def oracle_sample_inputs(n_ins: int, n_flows_q: int, rank: int):
    import workloads as wl
    out = []
    for idx, s in enumerate(SWEEP):
        ins, dels, flows = wl.flows_with_deletes(n_ins, N_FLOWS, s, DEL_FRAC, seed=seed_for(rank, idx), device="cpu")
        out.append((ins.numpy(), dels.numpy(), flows[:n_flows_q].numpy()))
    return out


def oracle_step(samples):
    import numpy as np
    import oracle
    n = 0
    answers = []
    for ins, dels, flows in samples:
        o = oracle.Sketch(D, W, Z, KB, SEED0)
        o.update(ins, np.ones(len(ins), np.int8), S=S)
        o.update(dels, -np.ones(len(dels), np.int8), S=S)
        answers.append(o.query(flows))
        n += len(ins) + len(dels) + len(flows)
    return n, answers


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    n_ins = args.ref_inserts
    samples = oracle_sample_inputs(n_ins, args.ref_queries, rank)
    for _ in range(args.warmup):
        oracle_step(samples)
    t0 = time.perf_counter()
    n = 0
    for _ in range(args.steps):
        k, _ = oracle_step(samples)
        n += k
    dt = time.perf_counter() - t0
    value = n / dt / 1e6
    sample = (f"per step, for each s in {list(SWEEP)}: the first {n_ins} of the 32,000,000 inserts, "
              f"10% of them deleted, {args.ref_queries} flows queried (same recipe and seeds)")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "M ops/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "flows-zipf-sweep-with-deletes (sampled)", "d": D, "w": W, "z": Z,
                       "key_bytes": KB, "chunk": S},
            "cpu_baseline": {"value": round(value, 4), "unit": "M ops/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "M ops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ref-inserts", type=int, default=400_000)
    ap.add_argument("--ref-queries", type=int, default=20_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="flows: skip the chunked-vs-sequential accuracy report (its one-at-a-time runs launch "
                         "thousands of kernels)")
    ap.add_argument("--workload", choices=["all", "flows", "batch", "serve", "accuracy", "pipeline", "profile",
                                           "l2curve", "seq", "outofl2", "batchprof", "rounds-accuracy"],
                    default="all",
                    help="all: the flows line with the batched and serving results embedded; profile: the small "
                         "fixed case the committed ncu summaries capture (two insert launches, the second profiled)")
    ap.add_argument("--profile-zipf", type=float, default=0.0)
    ap.add_argument("--flows-mode", choices=["single", "batched"], default="single",
                    help="flows step: one insert and one delete call per sketch (the single-sketch path, "
                         "default) or one batched launch over the six sketches per call")
    ap.add_argument("--print-kernel-sha", action="store_true",
                    help="print the chunk kernel's source hash (the key of the committed traffic record) and exit")
    ap.add_argument("--profile-inserts", type=int, default=2_000_000)
    ap.add_argument("--batch-sketches", type=int, default=1024)
    ap.add_argument("--batchprof-rounds", type=int, default=4,
                    help="batchprof: round count of the captured group (the autotuner's choice on this batch)")
    ap.add_argument("--serve-seconds", type=float, default=6.0, help="serve: seconds of each open-loop load (70 %%, 90 %%)")
    ap.add_argument("--ool2-updates", type=int, default=1_000_000_000,
                    help="outofl2: stream length (10^9 in the measured configuration)")
    args = ap.parse_args()
    if args.print_kernel_sha:
        print(chunk_kernel_source_sha256())
        return 0
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_env()

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    if args.impl == "reference":
        rc = run_reference(args, world, rank)
        if dist is not None:
            dist.destroy_process_group()
        return rc

    import numpy as np
    import paper_1701_04148_gb300 as sf
    import workloads as wl

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the SF-sketch library has no CPU path)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    L = sf.load()
    # One created stream for all of the bench's torch work and sketch calls, made current so that
    # they stay ordered; no implicit synchronisation with other work, as on the legacy default stream.
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)

    # the measurement kernels (roofline denominators) come from their own library
    ctx = dict(world=world, rank=rank, local=local, dist=dist, dev=dev, L=L, B=sf.load_bench(), stream=stream)
    line = None
    if args.workload in ("all", "flows"):
        line = run_flows(args, ctx)
    if args.workload in ("all", "batch"):
        b = run_batch(args, ctx)
        if line is None:
            line = b
        elif rank == 0:
            line["batched"] = b
    if args.workload == "accuracy":
        line = run_accuracy(args, ctx)
    if args.workload == "rounds-accuracy":
        line = run_rounds_accuracy(args, ctx)
    if args.workload == "pipeline":
        line = run_pipeline(args, ctx)
    if args.workload == "profile":
        line = run_profile(args, ctx)
    if args.workload == "batchprof":
        line = run_batch_profile(args, ctx)
    if args.workload == "l2curve":
        line = run_l2curve(args, ctx)
    if args.workload in ("all", "outofl2"):
        v = run_outofl2(args, ctx)
        if line is None:
            line = v
        elif rank == 0:
            line["out_of_l2"] = v
    if args.workload in ("all", "seq"):
        v = run_seq(args, ctx)
        if line is None:
            line = v
        elif rank == 0:
            line["one_at_a_time"] = v
    if args.workload in ("all", "serve"):
        v = run_serve(args, ctx)
        if line is None:
            line = v
        elif rank == 0:
            line["serving"] = v
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_flows(args, ctx):
    """The 5-tuple workload (the headline): Zipf sweep, inserts, deletes, Slim export, queries."""
    import numpy as np
    import torch

    import paper_1701_04148_gb300 as sf
    import workloads as wl
    world, rank, local, dist = ctx["world"], ctx["rank"], ctx["local"], ctx["dist"]
    dev, L, stream = ctx["dev"], ctx["L"], ctx["stream"]
    # ---- inputs, resident in HBM ----------------------------------------------------------
    inputs = []
    for idx, s in enumerate(SWEEP):
        ins, dels, flows = wl.flows_with_deletes(N_INS, N_FLOWS, s, DEL_FRAC, seed=seed_for(rank, idx), device=dev)
        inputs.append((ins, dels, flows))
    torch.cuda.synchronize()
    sketches = [sf.Sketch(D, W, Z, KB, SEED0, S, stream=stream) for _ in SWEEP]
    slims = [torch.empty(D * W, dtype=torch.int32, device=dev) for _ in SWEEP]
    answers = [torch.empty(N_FLOWS, dtype=torch.int32, device=dev) for _ in SWEEP]
    n_del = inputs[0][1].shape[0]
    ops_per_step = len(SWEEP) * (N_INS + n_del + N_FLOWS)
    # single mode: each sketch gets its own insert call and delete call (the single-sketch path);
    # batched mode: the sketches of the sweep are independent, so each update call can also be one
    # batched launch over all of them (same per-sketch semantics; see the batched-update tests)
    batched = args.flows_mode == "batched"
    del_ops = [torch.full((n_del,), -1, dtype=torch.int8, device=dev) for _ in SWEEP]
    slots = len(SWEEP) * ((S + 31) // 32 * 32)
    b_ins = sf.Batch(len(SWEEP), graph=True, stream=stream, max_round_slots=slots)
    b_del = sf.Batch(len(SWEEP), graph=True, stream=stream, max_round_slots=slots)
    # update launches plus a query per sketch
    launches_per_step = (2 if batched else 2 * len(SWEEP)) + len(SWEEP)

    pipe = None  # the sf.Pipeline of the pipelined host form

    def step(evs=None, host=None, direct=False, pipelined=False):
        """One step.  host: pinned host copies of the inputs (and answer buffers).  direct=False
        copies them to the device first and the answers back; direct=True hands the pinned host
        buffers to the same calls, and the kernels read the keys and write the answers over the
        host link themselves; pipelined=True updates each sketch through one sf_update_pipeline
        pipeline kept across the step (host keys copied in chunk-aligned pieces, overlapped with
        the updates and across calls) and queries with the host keys and answers directly."""
        src, out = inputs, answers
        if pipelined:
            for idx, sk in enumerate(sketches):
                sk.reset()
            if evs is not None:
                evs[0].record(stream)
            for idx, sk in enumerate(sketches):
                sk.update_through(pipe, host[idx][0], None, 1)
                sk.update_through(pipe, host[idx][1], None, -1)
            if evs is not None:
                evs[2].record(stream)
            hdrs = [sketches[idx].export_slim(slims[idx])[1] for idx in range(len(SWEEP))]
            for idx in range(len(SWEEP)):
                sf.query(slims[idx], hdrs[idx], host[idx][2], out=host[idx][3], stream=stream)
            if evs is not None:
                evs[4].record(stream)
            return
        if host is not None and not direct:
            for idx in range(len(SWEEP)):
                ins_h, dels_h, flows_h, _ = host[idx]
                ins_d, dels_d, flows_d = inputs[idx]
                ins_d.copy_(ins_h, non_blocking=True)
                dels_d.copy_(dels_h, non_blocking=True)
                flows_d.copy_(flows_h, non_blocking=True)
        elif host is not None:
            src = [(h[0], h[1], h[2]) for h in host]
            out = [h[3] for h in host]
        for sk in sketches:
            sk.reset()
        if evs is not None:
            evs[0].record(stream)
        if batched:
            b_ins.update([(sk, inp[0], None) for sk, inp in zip(sketches, src)])
        else:
            for sk, inp in zip(sketches, src):
                sk.insert(inp[0])
        if evs is not None:
            evs[1].record(stream)
        if batched:
            b_del.update([(sk, inp[1], o) for sk, inp, o in zip(sketches, src, del_ops)])
        else:
            for sk, inp in zip(sketches, src):
                sk.delete(inp[1])
        if evs is not None:
            evs[2].record(stream)
        hdrs = [sketches[idx].export_slim(slims[idx])[1] for idx in range(len(SWEEP))]
        if evs is not None:
            evs[3].record(stream)
        for idx in range(len(SWEEP)):
            sf.query(slims[idx], hdrs[idx], src[idx][2], out=out[idx], stream=stream)
        if evs is not None:
            evs[4].record(stream)
        if host is not None and not direct:
            for idx in range(len(SWEEP)):
                host[idx][3].copy_(answers[idx], non_blocking=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for sk in sketches:
        sk.sync()
    assert b_ins.sync_status() == sf.SF_OK and b_del.sync_status() == sf.SF_OK

    # ---- timed region (device-resident inputs) --------------------------------------------
    evs_all = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(gpu_index_for(local))
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(args.steps):
        step(evs_all[k])
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    for sk in sketches:
        sk.sync()
    t_ins = sum(evs_all[k][0].elapsed_time(evs_all[k][1]) for k in range(args.steps))
    t_del = sum(evs_all[k][1].elapsed_time(evs_all[k][2]) for k in range(args.steps))
    t_qry = sum(evs_all[k][2].elapsed_time(evs_all[k][4]) for k in range(args.steps))
    t_q_only = sum(evs_all[k][3].elapsed_time(evs_all[k][4]) for k in range(args.steps))
    ms_max = ms
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    value = world * ops_per_step / (ms_max / 1e3) / 1e6

    # ---- roofline denominators measured in this run, on a 64 MiB L2-resident buffer --------
    # The update issues as many read-modify-writes (Fat increments, Slim raises) as loads (Slim
    # minimum, Fat estimate), and on GB300 random L2 traffic of that 1:1 mix runs well below
    # either kind alone, so the peak is the measured rate of the mix (half the warps reduce, half
    # load); the load-only rate is reported beside it.
    best = l2_random_peaks(ctx["B"], dev, stream)
    upd_timed = args.steps * len(SWEEP) * (N_INS + n_del)
    chunk_ms = t_ins + t_del
    launches_chunk = args.steps * (2 if batched else 2 * len(SWEEP))
    achieved = upd_timed * L2_OPS_PER_UPDATE / (chunk_ms / 1e3) / 1e9
    tr = traffic_record()
    traffic = None
    rec_key = "flows_batched" if batched else "flows_single"
    if tr is not None and rec_key in tr:
        # DRAM bytes of this workload's own update launches (insert and delete launches of one step),
        # averaged per launch like `achieved`
        fb = tr[rec_key]
        traffic = round(fb["dram_bytes_per_step"] / fb["launches_per_step"])
    roofline = {"bound": "l2", "kernel": "chunk_update_kernel" if batched else "chunk_single_kernel",
                "achieved": round(achieved, 2),
                "peak": round(best["mix"], 2), "unit": "G random L2 ops/s", "frac": round(achieved / best["mix"], 4),
                "traffic": traffic,
                "peak_source": "measured in this run: random 32-bit ops on a 64 MiB L2-resident buffer, 1:1 "
                               "read-modify-write / load mix (the update's own mix)",
                "peak_red_only": round(best["red"], 2), "frac_of_red_only": round(achieved / best["red"], 4),
                "peak_load_only": round(best["ld"], 2), "frac_of_load_only": round(achieved / best["ld"], 4),
                "ops_per_update": L2_OPS_PER_UPDATE,
                "avg_launch_ms": round(chunk_ms / launches_chunk, 4)}
    # queries: d random gathers from an L2-resident Slim (4 MiB) per key, against the measured
    # random-load rate; the six query launches of a step are timed together (1 M keys each)
    gathers = args.steps * len(SWEEP) * N_FLOWS * L2_OPS_PER_QUERY
    roofline_query = {"bound": "l2", "kernel": "query_kernel",
                      "achieved": round(gathers / (t_q_only / 1e3) / 1e9, 2), "peak": round(best["ld"], 2),
                      "unit": "G random L2 ops/s", "frac": round(gathers / (t_q_only / 1e3) / 1e9 / best["ld"], 4),
                      "M_queries_per_s": round(args.steps * len(SWEEP) * N_FLOWS / t_q_only / 1e3, 1),
                      "avg_launch_us": round(t_q_only * 1e3 / (args.steps * len(SWEEP)), 2),
                      "note": f"{L2_OPS_PER_QUERY} Slim gathers per query (Sec. 3.1 query) over 1,000,000 13-byte "
                              f"keys per launch; peak: random 32-bit loads on 64 MiB in this run"}
    peaks, psrc = measured_peaks()
    hbm_bytes = upd_timed * (KB + L2_OPS_PER_UPDATE * 4)
    roofline_hbm = {"bound": "hbm", "achieved": round(hbm_bytes / (chunk_ms / 1e3) / 1e9, 1),
                    "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                    "frac": round(hbm_bytes / (chunk_ms / 1e3) / 1e9 / peaks.get("hbm_gbs", 1.0), 4),
                    "note": f"algorithmic bytes = key + 4 B per counter touched; peak {psrc}"}

    # ---- e2e: host pinned inputs, H2D + path + D2H of the answers inside the timed region ---
    e2e = None
    if not args.no_e2e:
        host = []
        for ins, dels, flows in inputs:
            host.append((ins.cpu().pin_memory(), dels.cpu().pin_memory(), flows.cpu().pin_memory(),
                         torch.empty(N_FLOWS, dtype=torch.int32).pin_memory()))
        h2d = sum(h[0].numel() + h[1].numel() + h[2].numel() for h in host)
        d2h = sum(h[3].numel() * 4 for h in host)

        pipe = sf.Pipeline(staging_bytes=2 * ((1 << 22) * KB + 16), device=dev)

        def timed_e2e(direct, pipelined=False):
            step(host=host, direct=direct, pipelined=pipelined)
            torch.cuda.synchronize()
            if dist is not None:
                dist.barrier()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            pev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
            a.record(stream)
            for k in range(args.steps):
                step(evs=pev[k], host=host, direct=direct, pipelined=pipelined)
            b.record(stream)
            torch.cuda.synchronize()
            ems = a.elapsed_time(b) / args.steps
            upd_ms = sum(pev[k][0].elapsed_time(pev[k][2]) for k in range(args.steps)) / args.steps
            rest_ms = sum(pev[k][2].elapsed_time(pev[k][4]) for k in range(args.steps)) / args.steps
            if dist is not None:
                t = torch.tensor([ems], dtype=torch.float64, device=dev)
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                ems = float(t.item())
            for sk in sketches:
                sk.sync()
            pipe.release_inputs()
            return {"value": round(world * ops_per_step / (ems / 1e3) / 1e6, 2), "unit": "M ops/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": round(ems, 3),
                    "update_ms_per_step": round(upd_ms, 3), "export_query_ms_per_step": round(rest_ms, 3)}

        ref_answers = [a.cpu() for a in answers]

        def link_gbps():
            """The host link's rate just now: one plain copy of sketch 0's pinned insert keys (416 MB)
            to its device buffer (the same bytes)."""
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            inputs[0][0].copy_(host[0][0], non_blocking=True)
            b.record(stream)
            torch.cuda.synchronize()
            return host[0][0].numel() / a.elapsed_time(b) / 1e6

        # A host form's time can differ from one repetition to the next, so the three forms run
        # interleaved, E2E_REPETITIONS times each, each repetition preceded by a plain copy that
        # records the host link's rate; each form reports its median repetition.
        forms = {"pipelined": (False, True), "direct": (True, False), "staged": (False, False)}
        reps = {k: [] for k in forms}
        links = {k: [] for k in forms}
        equal = {k: True for k in forms}
        def one_round():
            for name, (direct, pipelined) in forms.items():
                links[name].append(round(link_gbps(), 1))
                for h in host:
                    h[3].fill_(-1)
                reps[name].append(timed_e2e(direct, pipelined=pipelined))
                equal[name] &= all(torch.equal(host[i][3], ref_answers[i]) for i in range(len(SWEEP)))

        for _ in range(E2E_REPETITIONS):
            one_round()
        spread = max(max(x["ms_per_step"] for x in v) / min(x["ms_per_step"] for x in v) for v in reps.values())
        if spread > E2E_SPREAD:
            for _ in range(E2E_EXTRA):
                one_round()

        def median_rep(name):
            r = dict(sorted(reps[name], key=lambda x: x["ms_per_step"])[len(reps[name]) // 2])
            r["repetitions_ms_per_step"] = [x["ms_per_step"] for x in reps[name]]
            r["link_GBps_before_each"] = links[name]
            # the answers the host received equal the device-resident run's (same inputs)
            r["answers_equal_device_resident"] = equal[name]
            return r

        e2e = median_rep("pipelined")
        e2e["transfer"] = ("sf_update_pipeline per sketch and call through one pipeline kept across the "
                           "step: pinned host keys copied in chunk-aligned pieces of 2^22 keys into two "
                           "alternating staging halves on a copy stream, overlapped with the updates, each "
                           "call's first copy with the previous call's last update; the query kernel reads "
                           "the pinned flow keys and writes the answers to pinned host memory")
        e2e["measurement"] = (f"median of {len(reps['pipelined'])} repetitions of --steps steps ({E2E_REPETITIONS}, "
                              f"{E2E_REPETITIONS + E2E_EXTRA} when a form's repetitions differed by more than "
                              f"{E2E_SPREAD}x), the three forms interleaved; "
                              "link_GBps_before_each: a plain 416 MB pinned host-to-device copy timed just "
                              "before each repetition")
        direct_ = median_rep("direct")
        direct_["transfer"] = ("pinned host buffers passed to the same calls: the update calls copy the keys in "
                               "pieces of whole chunks into the idle half of each sketch's dictionary region "
                               "on a copy stream of the sketch's own, each piece applied while the next is "
                               "copied; the query kernel reads the pinned flow keys and writes the answers to "
                               "host memory")
        e2e["direct"] = direct_
        staged = median_rep("staged")
        staged["transfer"] = "cudaMemcpyAsync of the keys to device buffers, kernels, copy of the answers back"
        e2e["staged"] = staged

    # ---- both update forms on the same inputs, measured after the timed region -------------
    # single: one sf_insert_batch and one sf_delete_batch call per sketch (the single-sketch path);
    # batched: one batched launch over the six sketches per call.  Best of two passes each.
    single = batched_form = roofline_single = None
    if rank == 0:
        def per_sketch_pass():
            ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in SWEEP]
            for idx, sk in enumerate(sketches):
                sk.reset()
                ev[idx][0].record(stream)
                sk.insert(inputs[idx][0])
                ev[idx][1].record(stream)
                sk.delete(inputs[idx][1])
                ev[idx][2].record(stream)
            torch.cuda.synchronize()
            return ev

        def batched_pass():
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            for sk in sketches:
                sk.reset()
            ev[0].record(stream)
            b_ins.update([(sk, inp[0], None) for sk, inp in zip(sketches, inputs)])
            ev[1].record(stream)
            b_del.update([(sk, inp[1], o) for sk, inp, o in zip(sketches, inputs, del_ops)])
            ev[2].record(stream)
            torch.cuda.synchronize()
            return ev

        passes = [per_sketch_pass() for _ in range(2)]
        ev = min(passes, key=lambda e: sum(x[0].elapsed_time(x[2]) for x in e))
        ti = sum(e[0].elapsed_time(e[1]) for e in ev)
        td = sum(e[1].elapsed_time(e[2]) for e in ev)
        ins_ops = len(SWEEP) * N_INS * L2_OPS_PER_UPDATE / (ti / 1e3) / 1e9
        single = {"insert_mops": round(len(SWEEP) * N_INS / ti / 1e3, 1),
                  "delete_mops": round(len(SWEEP) * n_del / td / 1e3, 1),
                  "insert_mops_per_zipf_s": {str(x): round(N_INS / ev[i][0].elapsed_time(ev[i][1]) / 1e3, 1)
                                             for i, x in enumerate(SWEEP)},
                  "roofline_frac": round(len(SWEEP) * (N_INS + n_del) * L2_OPS_PER_UPDATE / ((ti + td) / 1e3) / 1e9
                                         / best["mix"], 4),
                  "note": "one sf_insert_batch / sf_delete_batch call per sketch, same inputs"}
        roofline_single = {
            "path": "C2 insert path: one sf_insert_batch of 32,000,000 13-byte keys per sketch (chunk 65,536, "
                    "d=4, w=2^18, z=16), the six Zipf exponents",
            "kernel": "chunk_single_kernel", "bound": "l2", "unit": "G random L2 ops/s",
            "ops_per_insert": L2_OPS_PER_UPDATE, "insert_G_per_s": round(len(SWEEP) * N_INS / ti / 1e6, 3),
            "achieved": round(ins_ops, 2), "peak": round(best["mix"], 2), "frac": round(ins_ops / best["mix"], 4),
            "peak_red_only": round(best["red"], 2), "frac_of_red_only": round(ins_ops / best["red"], 4),
            "peak_load_only": round(best["ld"], 2), "frac_of_load_only": round(ins_ops / best["ld"], 4),
            "peak_source": "measured in this run (sf_bench_random_access on 64 MiB): the 1:1 reduce/load mix, "
                           "RED.ADD alone and loads alone"}
        bpasses = [batched_pass() for _ in range(2)]
        bev = min(bpasses, key=lambda e: e[0].elapsed_time(e[2]))
        bi, bd = bev[0].elapsed_time(bev[1]), bev[1].elapsed_time(bev[2])
        batched_form = {"insert_mops": round(len(SWEEP) * N_INS / bi / 1e3, 1),
                        "delete_mops": round(len(SWEEP) * n_del / bd / 1e3, 1),
                        "updates_vs_single": round((ti + td) / (bi + bd), 3),
                        "note": "one batched launch over the six sketches per call (sf_batch_update), same inputs"}
        for sk in sketches:
            sk.sync()

    # ---- CPU baseline (the oracle) and a bit-exact check on the same bounded sample -------
    cpu = None
    exact = None
    if rank == 0 and not args.no_cpu_baseline:
        samples = []
        n_i = args.ref_inserts
        g_cpu = torch.Generator().manual_seed(SEED0)
        for idx in range(len(SWEEP)):
            ins, dels, flows = inputs[idx]
            head = ins[:n_i].cpu()
            victims = torch.randperm(n_i, generator=g_cpu)[: int(n_i * DEL_FRAC)]
            samples.append((head.numpy(), head[victims].contiguous().numpy(), flows[: args.ref_queries].cpu().numpy()))
        t0 = time.perf_counter()
        n_ops, want = oracle_step(samples)
        dt = time.perf_counter() - t0
        cpu = {"value": round(n_ops / dt / 1e6, 4), "unit": "M ops/s", "cores": 1, "kind": "oracle",
               "sample": f"for each s: first {args.ref_inserts} inserts, {int(args.ref_inserts * DEL_FRAC)} deletes, "
                         f"{args.ref_queries} queries of this run's inputs ({n_ops} ops, {dt:.1f} s)"}
        exact = True
        for idx, (ins_np, dels_np, fl_np) in enumerate(samples):
            g = sf.Sketch(D, W, Z, KB, SEED0, S, stream=stream)
            g.insert(torch.from_numpy(ins_np).to(dev))
            g.delete(torch.from_numpy(dels_np).to(dev))
            slim, hdr = g.export_slim()
            got = sf.query(slim, hdr, torch.from_numpy(fl_np).to(dev), stream=stream)
            g.sync()
            exact &= bool(np.array_equal(got.cpu().numpy().view(np.uint32), want[idx]))

    accuracy = accuracy_report(inputs, dev, stream) if rank == 0 and not args.no_accuracy else None
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "M ops/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "flows-zipf-sweep-with-deletes", "d": D, "w": W, "z": Z, "key_bytes": KB,
                       "chunk": S, "inserts_per_s": N_INS, "deletes_per_s": n_del, "flows": N_FLOWS,
                       "zipf_s": list(SWEEP), "l2": "inputs larger than L2 (2.7 GB of keys per step)",
                       "parallelism": f"replicas x{world}"},
            "breakdown": {"mode": ("the six sweep sketches updated by one batched launch per call" if batched else
                                   "one insert call and one delete call per sketch (the single-sketch path)"),
                          "insert_mops": round(args.steps * len(SWEEP) * N_INS / t_ins / 1e3, 1),
                          "delete_mops": round(args.steps * len(SWEEP) * n_del / t_del / 1e3, 1),
                          "export_query_mops": round(args.steps * len(SWEEP) * N_FLOWS / t_qry / 1e3, 1)},
            "roofline": roofline, "roofline_single_sketch": roofline_single, "roofline_hbm": roofline_hbm,
            "roofline_query": roofline_query, "single_sketch": single, "batched_form": batched_form,
            "cpu_baseline": cpu, "bit_exact_sample": exact, "e2e": e2e, "accuracy": accuracy,
            "gpu_launches": args.steps * launches_per_step, "clocks": clk,
        }
        return line
    return None


def accuracy_report(inputs, dev, stream, n_sample=8_000_000):
    """ARE / AAE of the chunked semantics (chunk 65,536) and of the paper's sequential semantics
    (chunk 1) against exact counts, per Zipf exponent, on the first n_sample inserts of each
    stream plus deletes of 10 % of those occurrences; all 1,000,000 flows are queried.
    RE = |f_hat - f| / f (Sec. 5.2); ARE averages it over flows with f > 0; AAE averages
    |f_hat - f| over all queried flows."""
    import torch

    import paper_1701_04148_gb300 as sf
    out = {}
    g_cpu = torch.Generator(device=dev)
    g_cpu.manual_seed(SEED0)
    for idx, s in enumerate(SWEEP):
        ins, _, flows = inputs[idx]
        head = ins[:n_sample]
        victims = torch.randperm(n_sample, generator=g_cpu, device=dev)[: int(n_sample * DEL_FRAC)]
        dels = head[victims].contiguous()
        # exact net counts of every flow (rows compared byte for byte)
        allk = torch.cat([flows, head, dels])
        _, inv = torch.unique(allk, dim=0, return_inverse=True)
        nf, nh, nd = flows.shape[0], head.shape[0], dels.shape[0]
        wts = torch.cat([torch.zeros(nf, dtype=torch.int64, device=dev), torch.ones(nh, dtype=torch.int64, device=dev),
                         -torch.ones(nd, dtype=torch.int64, device=dev)])
        cnt = torch.zeros(int(inv.max()) + 1, dtype=torch.int64, device=dev).index_add_(0, inv, wts)
        f = cnt[inv[:nf]]
        row = {}
        for name, S_ in (("chunk", S), ("seq", 1)):
            g = sf.Sketch(D, W, Z, KB, SEED0, S_, stream=stream)
            g.insert(head)
            g.delete(dels)
            slim, hdr = g.export_slim()
            est = sf.query(slim, hdr, flows, stream=stream).to(torch.int64) & 0xFFFFFFFF
            g.sync()
            err = (est - f).abs().to(torch.float64)
            present = f > 0
            row[f"are_{name}"] = float((err[present] / f[present].to(torch.float64)).mean())
            row[f"aae_{name}"] = float(err.mean())
            row[f"exact_frac_{name}"] = float((err[present] == 0).to(torch.float64).mean())
            assert bool((est >= f).all()), "under-estimation"
            g.close()
        out[str(s)] = {k: round(v, 5) for k, v in row.items()}
    return {"sample": f"first {n_sample} inserts of each s plus deletes of 10% of them; all {N_FLOWS} flows queried",
            "per_s": out}


def run_profile(args, ctx):
    """The small case of the chunk kernel that ncu captures: one sketch of the flows shape
    (d=4, w=2^18, z=16, 13-byte keys, chunk 65,536), `--profile-inserts` keys drawn with Zipf
    `--profile-zipf` over 10^6 flows; a warm-up insert launch, the profiled insert launch
    (launch index 1 of the chunk kernel), then deletes, export and queries.  Prints the
    CUDA-event time of the second insert launch."""
    import torch
    import paper_1701_04148_gb300 as sf
    import workloads as wl
    ins, dels, flows = wl.flows_with_deletes(args.profile_inserts, N_FLOWS, args.profile_zipf, DEL_FRAC,
                                             seed=2, device=ctx["dev"])
    g = sf.Sketch(D, W, Z, KB, 2, S)
    g.insert(ins)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx["stream"])
    g.insert(ins)
    e1.record(ctx["stream"])
    g.delete(dels)
    slim, hdr = g.export_slim()
    q = sf.query(slim, hdr, flows)
    st = g.sync_status()
    torch.cuda.synchronize()
    if st != sf.SF_OK:
        raise SystemExit(f"profile case failed: status {st}")
    ms = e0.elapsed_time(e1)
    g.close()
    return {"workload": "profile", "inserts": int(ins.shape[0]), "zipf": args.profile_zipf,
            "insert_ms": round(ms, 4), "M_inserts_per_s": round(ins.shape[0] / ms / 1e3, 1),
            "query_mean": float(q.to(torch.float64).mean())}


def run_batch_profile(args, ctx):
    """The small case of the batched update that ncu captures: one launch group of the many-sketch
    batch (the first sketches of the 1,024-sketch plan, in order, whose counters fit the default
    group budget of 3/4 of L2, as sf_batch_update groups them), chunks for R = --batchprof-rounds
    rounds (4 by default, what the autotuner picks for this batch on a GB300), one launch per call
    (group budget 0 on this subset), dictionaries in an arena.  A warm-up call, then the profiled call
    (launch index 1 of the chunk kernel)."""
    import torch
    import paper_1701_04148_gb300 as sf
    from paper_1701_04148_gb300 import autotune
    import workloads as wl
    dev, stream = ctx["dev"], ctx["stream"]
    plan = wl.many_sketch_plan(1024, seed=3)
    budget = torch.cuda.get_device_properties(dev).L2_cache_size * 3 // 4
    chunks_all = autotune.chunk_sizes([p["n"] for p in plan], args.batchprof_rounds)
    group, used = [], 0
    for p, c in zip(plan, chunks_all):
        fb = 4 * p["w"] * 16 * 4 + 4 * p["w"] * 4 + c * 32  # Fat + Slim + the dictionary a chunk touches
        if fb > budget:
            continue
        if used + fb > budget:
            break
        group.append((p, c))
        used += fb
    streams = []
    for p, _ in group:
        st, _ = wl.mixed_stream(p["n"], p["distinct"], p["s"], 0.1, 4, seed=p["seed"], device=dev)
        streams.append((st.keys, st.ops))
    sks = [sf.Sketch(4, p["w"], 16, 4, p["seed"], c, stream=stream, shared_dict=True) for p, c in group]
    slots = sum((c + 31) // 32 * 32 for _, c in group)
    # the dictionaries in an arena, as the bench's batched step has them (one launch: they fit)
    arena = sum(sf.dictionary_bytes(4, p["w"], 16, 4, p["seed"], c) for p, c in group)
    b = sf.Batch(len(sks), graph=False, stream=stream, max_round_slots=slots, group_bytes=0, dict_arena_bytes=arena)
    items = [(sk, k, o) for sk, (k, o) in zip(sks, streams)]
    b.update(items)
    for sk in sks:
        sk.reset()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.update(items)
    e1.record(stream)
    st = b.sync_status()
    torch.cuda.synchronize()
    if st != sf.SF_OK:
        raise SystemExit(f"batch profile case failed: status {st}")
    n = sum(p["n"] for p, _ in group)
    ms = e0.elapsed_time(e1)
    return {"workload": "batchprof", "rounds": args.batchprof_rounds, "sketches": len(group), "updates": n,
            "counter_bytes": used,
            "round_slots": slots, "launch_ms": round(ms, 4), "M_updates_per_s": round(n / ms / 1e3, 1)}


def run_seq(args, ctx):
    """The paper's one-at-a-time rule (chunk 1) on the insertion-only u32 workload: 100,000 keys
    Zipf(1.0) over 10,000 ids, d=4, w=4096, z=16; then all 10,000 ids queried.  GPU time of the
    insert call (best of --steps after --warmup), the CPU oracle's time for the same stream on one
    core, and a counter-by-counter check."""
    import numpy as np
    import torch

    import oracle
    import paper_1701_04148_gb300 as sf
    import workloads as wl
    dev, stream = ctx["dev"], ctx["stream"]
    keys, ids = wl.insert_only_u32(100_000, 10_000, 1.0, seed=1)
    kd, qd = keys.to(dev), ids.to(dev)
    g = sf.Sketch(4, 4096, 16, 4, 1, 1, stream=stream)
    for _ in range(args.warmup):
        g.reset()
        g.insert(kd)
    best = float("inf")
    for _ in range(args.steps):
        g.reset()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.insert(kd)
        b.record(stream)
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    slim, hdr = g.export_slim()
    est = sf.query(slim, hdr, qd, stream=stream)
    st = g.sync_status()
    o = oracle.Sketch(4, 4096, 16, 4, 1)
    t0 = time.perf_counter()
    o.update(keys.numpy(), np.ones(len(keys), np.int8), S=None)
    t_cpu = time.perf_counter() - t0
    exact = (st == sf.SF_OK
             and np.array_equal(g.fat.cpu().numpy().view(np.uint32).reshape(o.B.shape), o.B)
             and np.array_equal(slim.cpu().numpy().view(np.uint32).reshape(o.A.shape), o.A)
             and np.array_equal(est.cpu().numpy().view(np.uint32), o.query(ids.numpy())))
    return {"workload": "one-at-a-time-insert-u32", "updates": len(keys), "gpu_ms": round(best, 3),
            "gpu_M_updates_per_s": round(len(keys) / best / 1e3, 1), "oracle_ms_one_core": round(t_cpu * 1e3, 3),
            "speedup_vs_oracle": round(t_cpu * 1e3 / best, 2), "bit_exact": bool(exact)}


OOL2_D, OOL2_W, OOL2_Z, OOL2_KB, OOL2_S = 4, 1 << 22, 16, 8, 1 << 20
OOL2_DISTINCT, OOL2_ZIPF, OOL2_DEL, OOL2_SEED, OOL2_QUERIES = 1 << 26, 1.2, 0.2, 5, 1 << 24
OOL2_SECTOR = 32   # bytes one random counter access moves between L2 and HBM


def hbm_random_peaks(L, dev, stream, words=1 << 28):
    """Best of three rates (G ops/s) of sf_bench_random_access on a 1 GiB buffer (far beyond L2):
    32-bit loads (kind 2), reductions (kind 0) and the 1:1 reduce/load mix (kind 5)."""
    import torch
    buf = torch.zeros(words, dtype=torch.int32, device=dev)
    h_st = int(stream.cuda_stream)
    out = {}
    for name, kind in (("ld", 2), ("red", 0), ("mix", 5)):
        L.sf_bench_random_access(buf.data_ptr(), buf.numel(), 1 << 26, kind, 0, h_st)
        best = 0.0
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rc = L.sf_bench_random_access(buf.data_ptr(), buf.numel(), 1 << 28, kind, 0, h_st)
            b.record(stream)
            torch.cuda.synchronize()
            if rc != 0:
                raise SystemExit(f"sf_bench_random_access failed: {rc}")
            best = max(best, (1 << 28) / a.elapsed_time(b) / 1e6)
        out[name] = best
    del buf
    return out


def run_outofl2(args, ctx):
    """The out-of-L2 stress configuration: 10^9 u64 keys drawn Zipf(1.2) over 2^26 distinct ids,
    an 80/20 strict-turnstile insert/delete mix (each delete removes an earlier inserted
    occurrence), d=4, Fat 4 x 2^26 u32 counters (1 GiB, beyond L2), Slim 4 x 2^22, chunk 2^20,
    the whole stream in one update call per step; then the Slim is exported and 2^24 keys are
    queried (half drawn from the stream, half random 64-bit ids).  `--ool2-updates` shrinks the
    stream for the small case an ncu capture takes (same shapes otherwise).

    value = (updates + queries) / step time.  Roofline: the Fat and the chunk dictionary live in
    HBM, so every counter access is a random 32-byte sector; the ceiling is the random-access
    rate of a 1 GiB buffer with the update's 1:1 read-modify-write / load mix, measured in the
    same run."""
    import numpy as np
    import torch

    import oracle
    import paper_1701_04148_gb300 as sf
    import workloads as wl
    world, rank, local, dist = ctx["world"], ctx["rank"], ctx["local"], ctx["dist"]
    dev, L, stream = ctx["dev"], ctx["L"], ctx["stream"]
    n = args.ool2_updates
    st, _ = wl.mixed_stream(n, OOL2_DISTINCT, OOL2_ZIPF, OOL2_DEL, OOL2_KB, seed=OOL2_SEED + 1000 * rank,
                            device=dev)
    keys, ops = st.keys, st.ops
    n_del = int((ops < 0).sum())
    gq = wl._gen(77 + rank, dev)
    nq = OOL2_QUERIES
    pos = torch.randint(0, n, (nq // 2,), generator=gq, device=dev)
    absent = wl.ids_to_bytes(wl.distinct_ids(nq - nq // 2, 64, gq, dev), OOL2_KB)
    q = torch.cat([keys.index_select(0, pos), absent])
    q = q[torch.randperm(nq, generator=gq, device=dev)].contiguous()
    del pos, absent
    torch.cuda.synchronize()
    g = sf.Sketch(OOL2_D, OOL2_W, OOL2_Z, OOL2_KB, OOL2_SEED, OOL2_S, stream=stream)
    slim_buf = torch.empty(OOL2_D * OOL2_W, dtype=torch.int32, device=dev)
    ans = torch.empty(nq, dtype=torch.int32, device=dev)

    def step(evs=None, src=None, pipe=None):
        k, o, qq, out = src if src is not None else (keys, ops, q, ans)
        g.reset()
        if evs is not None:
            evs[0].record(stream)
        if pipe is not None:
            g.update_through(pipe, k, o)
        else:
            g.update(k, o)
        if evs is not None:
            evs[1].record(stream)
        slim, hdr = g.export_slim(slim_buf)
        if evs is not None:
            evs[2].record(stream)
        sf.query(slim, hdr, qq, out=out, stream=stream)
        if evs is not None:
            evs[3].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    g.sync()
    evs_all = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(gpu_index_for(local))
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(args.steps):
        step(evs_all[k])
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    g.sync()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = ms
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    t_upd = sum(e[0].elapsed_time(e[1]) for e in evs_all) / args.steps
    t_qry = sum(e[1].elapsed_time(e[3]) for e in evs_all) / args.steps
    t_q_only = sum(e[2].elapsed_time(e[3]) for e in evs_all) / args.steps
    value = world * (n + nq) / (ms_max / 1e3) / 1e6

    # Roofline.  Algorithmic bytes per update, every Fat access a random 32-byte sector of HBM
    # (the Slim, 64 MiB, counted as L2-resident): the key and op byte, d Fat increments (sector
    # read and write back) and the read-back: d sectors for an insertion's estimate, d 64-byte
    # buckets for a deletion's maximum.  Peak: the measured streaming copy rate.  The DRAM bytes
    # the kernel really moves come from an ncu capture of a 16-chunk prefix of the same stream,
    # scaled to this launch; as 32-byte sectors per second they are set against the random-access
    # rate of a 1 GiB buffer (the 1:1 reduce / load mix), measured in this run.
    n_ins = n - n_del
    alg_bytes = n_ins * (OOL2_KB + 1 + OOL2_D * 3 * OOL2_SECTOR) + n_del * (OOL2_KB + 1 + OOL2_D * 4 * OOL2_SECTOR)
    peaks, psrc = measured_peaks()
    achieved = alg_bytes / (t_upd / 1e3) / 1e9
    peaks_r = hbm_random_peaks(ctx["B"], dev, stream)
    tr = traffic_record("chunk_update_kernel_traffic.json")
    traffic = None
    if tr is not None and "outofl2" in tr:
        rec = tr["outofl2"]
        traffic = round((rec["dram_bytes_read"] + rec["dram_bytes_write"]) / rec["updates"] * n)
    roofline = {"bound": "hbm", "kernel": "chunk_update_kernel", "achieved": round(achieved, 1),
                "peak": peaks.get("hbm_gbs"), "unit": "GB/s", "frac": round(achieved / peaks.get("hbm_gbs", 1.0), 4),
                "traffic": traffic,
                "counting": f"algorithmic bytes per update: key + op byte + d Fat read-modify-writes "
                            f"(2 x {OOL2_SECTOR} B) + d Fat read-backs ({OOL2_SECTOR} B per insertion, "
                            f"{2 * OOL2_SECTOR} B bucket per deletion); {alg_bytes / n:.1f} B per update here",
                "peak_source": f"{psrc} streaming copy rate (MEASURED_PEAKS hbm_gbs)" if psrc == "measured"
                               else "fallback streaming copy rate",
                "avg_launch_ms": round(t_upd, 3)}
    if traffic is not None:
        # the key and op stream is read sequentially; the rest of the DRAM traffic is random sectors
        sect = (traffic - n * (OOL2_KB + 1)) / OOL2_SECTOR / (t_upd / 1e3) / 1e9
        roofline["dram_sectors"] = {
            "achieved_g_per_s": round(sect, 2), "peak_g_per_s": round(peaks_r["mix"], 2),
            "frac": round(sect / peaks_r["mix"], 4),
            "note": "DRAM bytes the kernel moves (ncu, scaled) less the sequential key and op stream, as 32-byte "
                    "sectors per second, against random 32-bit ops on a 1 GiB buffer (sf_bench_random_access kind "
                    "5, 1:1 reduce / load) in this run; that rate itself varied between 31 and 36 G/s across runs"}
    roofline["random_hbm_rates_g_ops"] = {k: round(v, 2) for k, v in peaks_r.items()}
    # queries: d random gathers per key from the exported 64 MiB Slim, against random 32-bit loads
    # on a 64 MiB buffer (measured in this run)
    ld64 = l2_random_peaks(ctx["B"], dev, stream)["ld"]
    g_q = nq * OOL2_D / (t_q_only / 1e3) / 1e9
    roofline_query = {"bound": "l2", "kernel": "query_kernel", "achieved": round(g_q, 2), "peak": round(ld64, 2),
                      "unit": "G random L2 ops/s", "frac": round(g_q / ld64, 4),
                      "M_queries_per_s": round(nq / t_q_only / 1e3, 1), "launch_us": round(t_q_only * 1e3, 1),
                      "note": f"{OOL2_D} gathers per query from the 64 MiB Slim; 8-byte keys"}

    # ---- e2e: keys, ops and queries in pinned host memory, answers written back to it --------
    e2e = None
    if not args.no_e2e:
        host = (keys.cpu().pin_memory(), ops.cpu().pin_memory(), q.cpu().pin_memory(),
                torch.empty(nq, dtype=torch.int32).pin_memory())
        # pieces of four chunks (2^22 updates of 8-byte keys and their operations) per staging half
        pipe = sf.Pipeline(staging_bytes=2 * (4 * OOL2_S * (OOL2_KB + 1) + 32), device=dev)
        ref = ans.cpu()

        def timed(use_pipe):
            host[3].fill_(-1)
            step(src=host, pipe=pipe if use_pipe else None)
            torch.cuda.synchronize()
            if dist is not None:
                dist.barrier()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(args.steps):
                step(src=host, pipe=pipe if use_pipe else None)
            b.record(stream)
            torch.cuda.synchronize()
            g.sync()
            pipe.release_inputs()
            ems = a.elapsed_time(b) / args.steps
            if dist is not None:  # the slowest rank's time
                t = torch.tensor([ems], dtype=torch.float64, device=dev)
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                ems = float(t.item())
            return ems, bool(torch.equal(host[3], ref))

        # the two host forms interleaved, E2E_REPETITIONS each; each reports its median repetition
        reps = {True: [], False: []}
        for _ in range(E2E_REPETITIONS):
            for use_pipe in (True, False):
                reps[use_pipe].append(timed(use_pipe))

        def form(use_pipe, transfer):
            ms_all = [r[0] for r in reps[use_pipe]]
            ems = sorted(ms_all)[E2E_REPETITIONS // 2]
            return {"value": round(world * (n + nq) / (ems / 1e3) / 1e6, 2), "unit": "M ops/s",
                    "h2d_bytes_per_step": int(host[0].numel() + host[1].numel() + host[2].numel()),
                    "d2h_bytes_per_step": int(host[3].numel() * 4), "ms_per_step": round(ems, 3),
                    "repetitions_ms_per_step": [round(x, 3) for x in ms_all], "transfer": transfer,
                    "answers_equal_device_resident": all(r[1] for r in reps[use_pipe])}

        e2e = form(True, "the update through an sf_pipeline (pinned keys and operations copied in pieces of four "
                         "chunks on a copy stream, overlapped with the updates); the query kernel reads the "
                         "pinned query keys and writes the answers to pinned host memory")
        e2e["direct"] = form(False, "pinned host buffers passed to the same calls (kernels read keys and ops and "
                                    "write the answers over the host link)")
        pipe.close()
        del host

    # ---- CPU baseline and bit-exact check on the first two chunks ----------------------------
    cpu = exact = None
    if rank == 0 and not args.no_cpu_baseline:
        pre = min(n, 2 * OOL2_S)
        kh, oh = keys[:pre].cpu().numpy(), ops[:pre].cpu().numpy()
        o = oracle.Sketch(OOL2_D, OOL2_W, OOL2_Z, OOL2_KB, OOL2_SEED)
        t0 = time.perf_counter()
        o.update(kh, oh, S=OOL2_S)
        dt = time.perf_counter() - t0
        cpu = {"value": round(pre / dt / 1e6, 4), "unit": "M updates/s", "cores": 1, "kind": "oracle",
               "sample": f"the first {pre} updates of the stream (two chunks, {dt:.1f} s)"}
        g2 = sf.Sketch(OOL2_D, OOL2_W, OOL2_Z, OOL2_KB, OOL2_SEED, OOL2_S, stream=stream)
        g2.update(keys[:pre], ops[:pre])
        g2.sync()
        exact = bool(np.array_equal(g2.fat.cpu().numpy().view(np.uint32).reshape(o.B.shape), o.B)
                     and np.array_equal(g2.slim.cpu().numpy().view(np.uint32).reshape(o.A.shape), o.A))
        g2.close()
        del o
    if rank != 0:
        return None
    return {"metric": METRIC, "value": round(value, 2), "unit": "M ops/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "out-of-l2-stress", "d": OOL2_D, "w": OOL2_W, "z": OOL2_Z, "key_bytes": OOL2_KB,
                       "chunk": OOL2_S, "updates": n, "deletes": n_del, "distinct": OOL2_DISTINCT,
                       "zipf_s": OOL2_ZIPF, "queries": nq, "fat_bytes": OOL2_D * OOL2_W * OOL2_Z * 4,
                       "l2": f"inputs larger than L2 ({n * (OOL2_KB + 1) / 1e9:.1f} GB of keys and ops per step)",
                       "parallelism": f"replicas x{world}"},
            "breakdown": {"update_ms": round(t_upd, 3), "M_updates_per_s": round(n / t_upd / 1e3, 1),
                          "export_query_ms": round(t_qry, 3), "M_queries_per_s": round(nq / t_q_only / 1e3, 1)},
            "roofline": roofline, "roofline_query": roofline_query, "cpu_baseline": cpu,
            "bit_exact_first_two_chunks": exact, "e2e": e2e, "gpu_launches": args.steps * 2, "clocks": clk}


def run_l2curve(args, ctx):
    """Random 32-bit loads, reductions and the 1:1 mix (sf_bench_random_access kinds 2, 0, 5;
    2^28 operations, best of three) over buffers of 32-160 MiB: where the L2 stops holding a
    random working set; then the returning atomic forms (kinds 1, 3, 4, 6) at 64 MiB and 1 GiB."""
    import torch
    L, dev, stream = ctx["B"], ctx["dev"], ctx["stream"]
    mib = 1 << 20
    buf = torch.zeros((160 * mib) // 4, dtype=torch.int32, device=dev)
    h_st = int(stream.cuda_stream)
    rows = []
    for size in (32, 48, 56, 60, 64, 68, 72, 76, 80, 88, 96, 112, 128, 160):
        n = size * mib // 4
        row = {"mib": size}
        for name, kind in (("ld", 2), ("red", 0), ("mix", 5)):
            L.sf_bench_random_access(buf.data_ptr(), n, 1 << 26, kind, 0, h_st)
            best = 0.0
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                rc = L.sf_bench_random_access(buf.data_ptr(), n, 1 << 28, kind, 0, h_st)
                b.record(stream)
                torch.cuda.synchronize()
                if rc != 0:
                    raise SystemExit(f"sf_bench_random_access failed: {rc}")
                best = max(best, (1 << 28) / a.elapsed_time(b) / 1e6)
            row[name] = round(best, 1)
        rows.append(row)
    # the returning forms (atomicAdd with its result used, 32-bit CAS) and atomicMax beside the
    # plain reduction, in L2 (64 MiB) and in HBM (1 GiB)
    atomics = []
    big = torch.zeros((1024 * mib) // 4, dtype=torch.int32, device=dev)
    for size, b in ((64, buf), (1024, big)):
        n = size * mib // 4
        row = {"mib": size}
        for name, kind in (("red", 0), ("atom_ret", 1), ("red_max", 3), ("cas32", 4), ("cas128", 6)):
            L.sf_bench_random_access(b.data_ptr(), n, 1 << 26, kind, 0, h_st)
            best = 0.0
            for _ in range(3):
                a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                rc = L.sf_bench_random_access(b.data_ptr(), n, 1 << 28, kind, 0, h_st)
                e.record(stream)
                torch.cuda.synchronize()
                if rc != 0:
                    raise SystemExit(f"sf_bench_random_access failed: {rc}")
                best = max(best, (1 << 28) / a.elapsed_time(e) / 1e6)
            row[name] = round(best, 1)
        atomics.append(row)
    del buf, big
    # one grid barrier of the persistent update kernel's kind (cooperative, one block per SM)
    scr = torch.zeros(64, dtype=torch.int32, device=dev)
    L.sf_bench_grid_barrier(scr.data_ptr(), 100, h_st)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    rc = L.sf_bench_grid_barrier(scr.data_ptr(), 2000, h_st)
    b.record(stream)
    torch.cuda.synchronize()
    if rc != 0:
        raise SystemExit(f"sf_bench_grid_barrier failed: {rc}")
    return {"workload": "l2curve", "unit": "G random 32-bit ops/s", "rows": rows, "atomics": atomics,
            "grid_barrier_us": round(a.elapsed_time(b) * 1e3 / 2000, 3)}


def run_rounds_accuracy(args, ctx):
    """What the batch autotuner's chunk sizes cost in accuracy: six sketches of the many-sketch plan
    (every 170th by stream length: 10^4 to 2.8 x 10^6 updates of the 90/10 turnstile mix, u32 keys,
    d=4, z=16), each updated one at a time (S = 1, the paper's rule) and in chunks of ceil(n / R) for
    the autotuner's round counts R; the average relative error of the point query over the ids with
    a positive count, against exact counts (a per-id sum of the stream's +1/-1)."""
    import torch

    import paper_1701_04148_gb300 as sf
    import workloads as wl
    dev, stream = ctx["dev"], ctx["stream"]
    plan = wl.many_sketch_plan(args.batch_sketches, seed=3)
    picked = sorted(plan, key=lambda p: p["n"])[::170][:6]
    rounds = (32, 16, 8, 4, 2)
    out = []
    for p in picked:
        st, ids = wl.mixed_stream(p["n"], p["distinct"], p["s"], 0.1, 4, seed=p["seed"], device=dev)
        kid = st.keys.view(torch.int32).view(-1).to(torch.int64) & 0xFFFFFFFF
        idv = ids.view(torch.int32).view(-1).to(torch.int64) & 0xFFFFFFFF
        srt, order = torch.sort(idv)
        where = order[torch.searchsorted(srt, kid)]
        true = torch.zeros(idv.numel(), dtype=torch.int64, device=dev)
        true.index_add_(0, where, st.ops.to(torch.int64))
        live = true > 0
        rec = {"n": p["n"], "w": p["w"], "zipf_s": round(p["s"], 3), "ids_live": int(live.sum())}
        for R in (None,) + rounds:
            S = 1 if R is None else min(1 << 20, max(2, -(-p["n"] // R)))  # as the autotuner clamps
            g = sf.Sketch(4, p["w"], 16, 4, p["seed"], S, stream=stream)
            g.update(st.keys, st.ops)
            slim, hdr = g.export_slim()
            est = sf.query(slim, hdr, ids, stream=stream).to(torch.int64) & 0xFFFFFFFF
            if g.sync_status() != sf.SF_OK:
                raise SystemExit("rounds-accuracy: update failed")
            are = ((est[live] - true[live]).abs().to(torch.float64) / true[live].to(torch.float64)).mean()
            rec["are_one_at_a_time" if R is None else f"are_R{R}"] = round(float(are), 5)
            g.close()
        out.append(rec)
    return {"workload": "rounds-accuracy", "rounds": list(rounds), "sketches": out,
            "note": "ARE of the point query over ids with a positive count; chunk = ceil(n / R), at most 2^20"}


def run_accuracy(args, ctx):
    """Accuracy experiments of Sec. 5.2 (uniform and skewed workloads) on synthetic stand-ins for
    the YCSB traces: d=5, w=40,000, z=3, 100,000 distinct items, 10,000,000 insertions drawn
    uniformly or Zipf(0.99), then deletion of the same insertions in reverse order.  Reports the
    fraction of items with RE < 1 % after the insertions (Fig. CDF-RE), ARE after every 1,000,000
    insertions and after every 1,000,000 deletions, for the paper's one-at-a-time semantics
    (chunk 1) and the chunked semantics (chunk 65,536).  The paper reports 74.51 % (uniform) and
    74.30 % (skewed) of items below 1 % RE for SF-sketch (Sec. 5.2.1, 5.2.2).  The same runs with
    the SF_4 deletion rule (Sec. 3.4: clamp to the bucket sum, not the maximum) give the ablation
    against SF_F: the insertion phase is identical, the deletion phase shows what SF_F's tighter
    bound buys."""
    import torch

    import paper_1701_04148_gb300 as sf
    import workloads as wl
    dev, stream = ctx["dev"], ctx["stream"]
    d, w, z, n_items, n_ins, step = 5, 40_000, 3, 100_000, 10_000_000, 1_000_000
    out = {"workload": "accuracy-sec5.2", "d": d, "w": w, "z": z, "items": n_items, "insertions": n_ins,
           "paper_re_below_1pct": {"uniform": 0.7451, "skewed": 0.7430}}
    for name, s_ in (("uniform", 0.0), ("skewed", 0.99)):
        keys, ids = wl.insert_only_u32(n_ins, n_items, s_, seed=7 if s_ == 0 else 8, device=dev)
        kid = keys.view(torch.int32).reshape(-1)
        idv = ids.view(torch.int32).reshape(-1)
        sid, order = torch.sort(idv)
        pos = order[torch.searchsorted(sid, kid)]           # item index of every insertion
        res = {}
        for sem, S_, rule in (("seq", 1, "sff"), ("chunk", 65536, "sff"), ("sf4_seq", 1, "sf4"),
                              ("sf4_chunk", 65536, "sf4")):
            g = sf.Sketch(d, w, z, 4, 11, S_, stream=stream, delete_rule=rule)
            f = torch.zeros(n_items, dtype=torch.int64, device=dev)
            are_ins, are_del = [], []

            def score():
                slim, hdr = g.export_slim()
                est = sf.query(slim, hdr, ids, stream=stream).to(torch.int64) & 0xFFFFFFFF
                present = f > 0
                re = (est - f).abs().to(torch.float64)[present] / f[present].to(torch.float64)
                assert bool((est >= f).all())
                return float(re.mean()), float((re < 0.01).to(torch.float64).mean())

            for b0 in range(0, n_ins, step):
                g.insert(keys[b0:b0 + step])
                f.index_add_(0, pos[b0:b0 + step], torch.ones(step, dtype=torch.int64, device=dev))
                are_ins.append(round(score()[0], 5))
            below = score()[1]
            for b1 in range(n_ins, 0, -step):                     # reverse order of the insertions
                b0 = b1 - step
                g.delete(keys[b0:b1].flip(0).contiguous())
                f.index_add_(0, pos[b0:b1], -torch.ones(step, dtype=torch.int64, device=dev))
                if b0 > 0:
                    are_del.append(round(score()[0], 5))
            g.sync()
            res[sem] = {"re_below_1pct": round(below, 4), "are_after_each_1M_insertions": are_ins,
                        "are_during_reverse_deletion": are_del}
            g.close()
        out[name] = res
    return out


def run_pipeline(args, ctx):
    """The paper's GPU query experiment (Sec. 4.2, 5.4) on this GPU: batches of b host keys go
    through sf_query_pipelined (split over n streams, copy in, query, copy out), b from 1 K to
    64 K.  Throughput: many batches back to back; latency: one batch alone, submit to answers in
    host memory.  The Slim is the Zipf(1.0) 5-tuple sketch (d=4, w=2^18).  Paper (Tesla C2075):
    ~50 Mqps at 20 K, >110 Mqps at 64 K, mean latency < 410 us up to 28 K."""
    import numpy as np
    import torch

    import paper_1701_04148_gb300 as sf
    import workloads as wl
    dev, stream = ctx["dev"], ctx["stream"]
    ins, dels, flows = wl.flows_with_deletes(N_INS, N_FLOWS, 1.0, DEL_FRAC, seed=SEED0 + 2, device=dev)
    g = sf.Sketch(D, W, Z, KB, SEED0, S, stream=stream)
    g.insert(ins)
    g.delete(dels)
    slim, hdr = g.export_slim()
    g.sync()
    del ins, dels
    n_streams = 4
    streams = [torch.cuda.Stream(device=dev) for _ in range(n_streams)]
    rows = []
    for b in (1024, 4096, 8192, 16384, 20000, 28000, 32768, 65536):
        kh = flows[:b].cpu().pin_memory()
        oh = torch.zeros(b, dtype=torch.int32).pin_memory()
        kd = torch.empty((b, KB), dtype=torch.uint8, device=dev)
        od = torch.empty(b, dtype=torch.int32, device=dev)
        for _ in range(5):
            sf.query_pipelined(slim, hdr, kh, oh, kd, od, streams)
        torch.cuda.synchronize()
        lat = []
        for _ in range(50):
            t = time.perf_counter()
            sf.query_pipelined(slim, hdr, kh, oh, kd, od, streams)
            for s_ in streams:
                s_.synchronize()
            lat.append(time.perf_counter() - t)
        reps = max(20, int(4_000_000 // b))
        t = time.perf_counter()
        for _ in range(reps):
            sf.query_pipelined(slim, hdr, kh, oh, kd, od, streams)
        for s_ in streams:
            s_.synchronize()
        dt = time.perf_counter() - t
        rows.append({"batch": b, "mqps": round(b * reps / dt / 1e6, 1),
                     "mean_latency_us": round(1e6 * float(np.mean(lat)), 1),
                     "p99_latency_us": round(1e6 * float(np.percentile(lat, 99)), 1)})
    return {"workload": "query-pipeline-sec4.2", "streams": n_streams, "key_bytes": KB, "rows": rows,
            "paper_tesla_c2075": {"mqps_at_20K": 50, "mqps_at_64K": 110, "mean_latency_us_upto_28K": 410}}


def run_batch(args, ctx):
    """Many-node update: --batch-sketches sketches (Slim widths log-uniform 2^10..2^16, Fat 16x, d=4,
    stream lengths log-uniform 10^4..10^7 u32 keys, Zipf s ~ U(0.5, 1.5), 90/10 insert/delete)
    in one persistent graph-captured launch per step (batched) versus one sf_update_batch call
    per sketch (plain), same chunk sizes (picked by the autotuner), same GPU."""
    import torch

    import paper_1701_04148_gb300 as sf
    from paper_1701_04148_gb300 import autotune, shard
    import workloads as wl
    world, rank, dist, dev, stream = ctx["world"], ctx["rank"], ctx["dist"], ctx["dev"], ctx["stream"]
    # one batch of independent sketches (monitoring nodes, Sec. 1.1) sharded over the ranks: each
    # rank updates the sketches shard.assign gives it (longest stream first onto the least-loaded
    # rank); no collective touches the data path, only the step time is reduced (max over ranks)
    plan_all = wl.many_sketch_plan(args.batch_sketches, seed=3)
    lengths_all = [p["n"] for p in plan_all]
    mine = shard.owned(lengths_all, world, rank)
    plan = [plan_all[i] for i in mine]
    total_all = sum(lengths_all)
    t0 = time.time()
    streams = []
    for p in plan:
        st, _ = wl.mixed_stream(p["n"], p["distinct"], p["s"], 0.1, 4, seed=p["seed"], device=dev)
        streams.append((st.keys, st.ops))
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    ns = [p["n"] for p in plan]
    ws = [p["w"] for p in plan]
    total = sum(ns)

    # SF_FLAG_SHARED_DICT sketches: the batch's launch groups, which run one after another, reuse one
    # dictionary arena (1/32 of device memory), and the plain per-sketch calls, one after another on
    # one stream, reuse one dictionary buffer
    arena_bytes = torch.cuda.get_device_properties(dev).total_memory // 32

    def make(chunks):
        return [sf.Sketch(4, w, 16, 4, p["seed"], S, stream=stream, shared_dict=True)
                for w, p, S in zip(ws, plan, chunks)]

    cache = os.path.join(ROOT, "paper_1701_04148_gb300", "_build", "autotune_cache.json")
    key = autotune.shape_key(ws, ns, 4, 16, 4) + "-" + torch.cuda.get_device_name(dev).replace(" ", "_")
    t1 = time.time()
    tuned = autotune.tune(make, streams, ns, cache_path=cache, cache_key=key, widths=ws, d=4, z=16,
                          dict_arena_bytes=arena_bytes)
    tune_s = time.time() - t1
    chunks = tuned["chunks"]
    bsk, psk = make(chunks), make(chunks)
    plain_dict = torch.empty(max(sf.dictionary_bytes(4, w, 16, 4, p["seed"], S) for w, p, S in zip(ws, plan, chunks)),
                             dtype=torch.uint8, device=dev)
    for sk in psk:
        sk.set_dictionary(plain_dict)
    batch = sf.Batch(len(bsk), graph=True, stream=stream, max_round_slots=tuned["round_slots"],
                     block_threads=tuned["block_threads"], group_bytes=tuned["group_bytes"],
                     dict_arena_bytes=arena_bytes)
    items = [(sk, k, o) for sk, (k, o) in zip(bsk, streams)]

    def batched_step():
        for sk in bsk:
            sk.reset()
        batch.update(items)

    def plain_step():
        for sk, (k, o) in zip(psk, streams):
            sk.reset()
            sk.update(k, o)

    for _ in range(args.warmup):
        batched_step()
    plain_step()
    torch.cuda.synchronize()

    def timed(fn, k):
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / k
        if dist is not None:
            t = torch.tensor([ms], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    tb = timed(batched_step, args.steps)
    tp = timed(plain_step, max(1, args.steps // 2))
    st_b = batch.sync_status()
    exact = all(torch.equal(a.fat, b.fat) and torch.equal(a.slim, b.slim) for a, b in zip(bsk, psk))
    info = batch.info()
    # roofline of this rank's batched step: each update makes 4d random counter accesses (L2 ops; the
    # launch groups keep each launch's counters within L2), against the 1:1 mix measured in this run;
    # and its algorithmic HBM bytes (key 4 B + op 1 B + 4 B per counter access) against the copy peak
    best = l2_random_peaks(ctx["B"], dev, stream)
    ops_s = total * L2_OPS_PER_UPDATE / (tb / 1e3) / 1e9
    tr = traffic_record("chunk_update_kernel_traffic.json")
    traffic = None
    # the captured group's chunks must be those of the tuned round count (DRAM bytes per update
    # grow with the chunk size: a larger chunk touches more dictionary)
    if tr is not None and "c3_group" in tr and info["groups_last"] and tr["c3_group"].get("rounds") == tuned["rounds"]:
        g = tr["c3_group"]
        traffic = round(g["dram_bytes"] / g["updates"] * total / info["groups_last"])
    roofline = {"bound": "l2", "kernel": "chunk_update_kernel", "achieved": round(ops_s, 2), "peak": round(best["mix"], 2),
                "unit": "G random L2 ops/s", "frac": round(ops_s / best["mix"], 4),
                "peak_red_only": round(best["red"], 2), "frac_of_red_only": round(ops_s / best["red"], 4),
                "peak_load_only": round(best["ld"], 2), "frac_of_load_only": round(ops_s / best["ld"], 4),
                "ops_per_update": L2_OPS_PER_UPDATE, "traffic": traffic,
                "traffic_note": "DRAM bytes per launch: one launch group's application-replay capture "
                                "(chunk_update_kernel_traffic.json, c3_group) scaled to this step's updates "
                                "and launch groups",
                "avg_launch_ms": round(tb / max(1, info["groups_last"]), 4)}
    hbm_b = total * (4 + 1 + L2_OPS_PER_UPDATE * 4)
    peaks, psrc = measured_peaks()
    roofline_hbm = {"bound": "hbm", "achieved": round(hbm_b / (tb / 1e3) / 1e9, 1), "peak": peaks.get("hbm_gbs"),
                    "unit": "GB/s", "frac": round(hbm_b / (tb / 1e3) / 1e9 / peaks.get("hbm_gbs", 1.0), 4),
                    "note": f"algorithmic bytes = 4 B key + 1 B op + 4 B per counter access ({4 + 1 + 4 * L2_OPS_PER_UPDATE} "
                            f"B per update); peak {psrc}"}
    out = {"workload": "batched-many-sketch", "metric": "M updates/s", "sketches": len(plan_all),
           "updates_per_step": total_all, "value": round(total_all / (tb / 1e3) / 1e6, 2), "unit": "M updates/s",
           "plain_value": round(total_all / (tp / 1e3) / 1e6, 2), "batched_vs_plain_speedup": round(tp / tb, 3),
           "ms_per_step_batched": round(tb, 3), "ms_per_step_plain": round(tp, 3), "rounds": tuned["rounds"],
           "block_threads": tuned["block_threads"], "group_bytes": tuned["group_bytes"],
           "autotune_updates_per_s": tuned["trials"], "autotune_block": tuned["trials_block"],
           "autotune_group": tuned["trials_group"], "autotune_best_rounds_bracketed": tuned["best_rounds_bracketed"],
           "autotune_rounds_skipped_for_memory": tuned["rounds_skipped_for_memory"],
           "sketch_bytes": autotune.sketch_bytes(ws, chunks, 4, 16, shared_dict=True),
           "dict_arena_bytes": arena_bytes,
           "sketch_bytes_with_own_dictionaries": autotune.sketch_bytes(ws, chunks, 4, 16),
           "graph": info, "status": st_b, "roofline": roofline, "roofline_hbm": roofline_hbm,
           "launch_groups": {"groups": info["groups_last"], "group_bytes": info["group_bytes"],
                             "rule": "sketches whose counters fit the budget packed into L2-sized launch "
                                     "groups, larger ones share one launch; a group whose dictionaries do "
                                     "not fit the arena together is split"},
           "batched_equals_plain": bool(exact), "gen_s": round(gen_s, 1), "autotune_s": round(tune_s, 1),
           "n_gpus": world, "scaling": "strong",
           "shard": {"ranks": world, "sketches_rank0": len(mine), "updates_rank0": total,
                     "imbalance": round(shard.imbalance(lengths_all, world), 4),
                     "rule": "the same 1,024-sketch batch on every N: each rank updates the sketches "
                             "shard.assign gives it (longest stream first), no data-path collective; "
                             "value = all updates / max step time over ranks"}}
    batch.close()
    for sk in bsk + psk:
        sk.close()
    del streams
    torch.cuda.empty_cache()
    return out


def run_serve(args, ctx):
    """Collector serving loop: 4,096 resident Slims (widths log-uniform 2^10..2^18, d=4) filled from
    u32 Zipf streams, a 40 GB admission budget, open-loop Poisson query batches of round(2^U(0,16))
    keys (80 % Zipf-hot present, 20 % uniform absent) at ~70 % and ~90 % of the measured capacity,
    with replace-in-place uploads during the runs; then a 1 GB budget where admission binds; and the plain
    path (one sf_query_batch per request, copies included) for comparison."""
    import threading

    import numpy as np
    import torch

    import paper_1701_04148_gb300 as sf
    import workloads as wl
    rank, dev, stream = ctx["rank"], ctx["dev"], ctx["stream"]
    n_sk = 4096
    g = torch.Generator().manual_seed(4 + 1000 * rank)
    widths = [wl.log_uniform_int(10.0, 18.0, g) for _ in range(n_sk)]
    # fill the Slims with the batched update, 256 sketches at a time, keep only the exported Slims
    slims, hdrs, idtabs = [], [], []
    t0 = time.time()
    for g0 in range(0, n_sk, 256):
        grp = list(range(g0, min(n_sk, g0 + 256)))
        sks, items = [], []
        for k in grp:
            w = widths[k]
            st, ids = wl.mixed_stream(2 * w, 4 * w, 1.0, 0.1, 4, seed=50_000 + k + 1000 * rank, device=dev)
            sk = sf.Sketch(4, w, 16, 4, 7 + k, 2048, stream=stream)
            sks.append(sk)
            items.append((sk, st.keys, st.ops))
            idtabs.append(ids.view(torch.int32).reshape(-1).cpu().numpy())
        b = sf.Batch(len(sks), stream=stream)
        b.update(items)
        b.sync()
        for sk in sks:
            slim, hdr = sk.export_slim()
            slims.append(slim)
            hdrs.append(hdr)
            sk.close()
        b.close()
        del sks, items
    torch.cuda.synchronize()
    build_s = time.time() - t0
    slim_bytes = sum(4 * 4 * w for w in widths)

    # request pool: 1024 pre-generated host key arrays
    rng = np.random.default_rng(11 + rank)
    pool = []
    for q in range(1024):
        k = int(rng.integers(n_sk))
        n = int(round(2 ** rng.uniform(0, 16)))
        ids = idtabs[k]
        n_hot = int(round(0.8 * n))
        ranks = np.minimum(rng.zipf(1.1, n_hot) - 1, len(ids) - 1)
        keys = np.concatenate([ids[ranks], rng.integers(0, 2**31, n - n_hot).astype(np.int32)])
        rng.shuffle(keys)
        pool.append((k, np.ascontiguousarray(keys), np.zeros(n, np.uint32)))
    mean_keys = float(np.mean([len(p[1]) for p in pool]))

    col = sf.Collector(budget_bytes=40 << 30, max_sketches=n_sk, n_streams=4, max_batch_keys=1 << 17,
                       max_batch_reqs=512, max_wait_us=50)
    for k in range(n_sk):
        assert col.upload(k, slims[k], hdrs[k]) == sf.SF_OK

    # capacity: closed loop, as fast as one client thread submits
    def burst(n_req):
        ts = []
        t = time.perf_counter()
        for q in range(n_req):
            k, keys, out = pool[q % len(pool)]
            ts.append(col.submit(k, keys, out))
        for x in ts:
            col.wait(x)
        return time.perf_counter() - t

    burst(256)
    col.stats(reset=True)
    dt = burst(4096)
    cap = col.stats(reset=True)
    cap_keys_s = cap["keys"] / dt

    # open loop at ~70 % and ~90 % of capacity: Poisson arrivals, replace-in-place uploads at 20/s
    def open_loop(frac, seconds, seed):
        rate = frac * cap_keys_s / mean_keys
        gaps = wl.poisson_gaps(int(rate * seconds) + 1, rate, torch.Generator().manual_seed(seed)).numpy()
        arrivals = np.cumsum(gaps)
        stop = threading.Event()
        uploads = [0]

        def uploader():
            r2 = np.random.default_rng(99 + seed)
            while not stop.is_set():
                k = int(r2.integers(n_sk))
                if col.upload(k, slims[k], hdrs[k]) == sf.SF_OK:
                    uploads[0] += 1
                time.sleep(0.05)

        th = threading.Thread(target=uploader)
        th.start()
        tickets = []
        t_start = time.perf_counter()
        for q, at in enumerate(arrivals):
            while True:
                now = time.perf_counter() - t_start
                if now >= at:
                    break
                if at - now > 2e-4:
                    time.sleep((at - now) - 1e-4)
            k, keys, out = pool[q % len(pool)]
            tickets.append(col.submit(k, keys, out))
        for x in tickets:
            col.wait(x)
        stop.set()
        th.join()
        st_ = col.stats(reset=True)
        return {"load_fraction_of_capacity": frac, "p50_ms": round(st_["p50_us"] / 1e3, 4),
                "p99_ms": round(st_["p99_us"] / 1e3, 4), "mean_ms": round(st_["mean_us"] / 1e3, 4),
                "queries_per_s": round(st_["qps"], 1),
                "offered_requests_per_s": round(len(arrivals) / (time.perf_counter() - t_start), 1),
                "requests": int(st_["requests"]), "uploads_during_run": uploads[0]}

    loads = [open_loop(0.7, args.serve_seconds, 5), open_loop(0.9, args.serve_seconds, 6)]
    open70 = loads[0]

    # check a sample of answers against sf_query_batch (alone) on the same Slims
    exact = True
    for q in range(0, len(pool), 97):
        k, keys, _ = pool[q]
        out = np.zeros(len(keys), np.uint32)
        col.wait(col.submit(k, keys, out))
        want = sf.query(slims[k], hdrs[k], torch.from_numpy(keys).to(dev)).cpu().numpy().view(np.uint32)
        exact &= bool(np.array_equal(out, want))
    col.close()

    # plain path: one sf_query_batch per request with its own copies, one at a time
    t = time.perf_counter()
    nk = 0
    for q in range(1024):
        k, keys, _ = pool[q]
        kd = torch.from_numpy(keys).to(dev, non_blocking=True)
        res = sf.query(slims[k], hdrs[k], kd).cpu()
        nk += len(keys)
    plain_keys_s = nk / (time.perf_counter() - t)

    # tight budget: admission binds
    tight = sf.Collector(budget_bytes=1 << 30, max_sketches=n_sk, n_streams=1)
    admitted = sum(1 for k in range(n_sk) if tight.upload(k, slims[k], hdrs[k]) == sf.SF_OK)
    tst = tight.stats()
    tight.close()
    return {"workload": "collector-serving", "sketches": n_sk, "slim_bytes": slim_bytes,
            "p50_ms": open70["p50_ms"], "p99_ms": open70["p99_ms"], "mean_ms": open70["mean_ms"],
            "queries_per_s": open70["queries_per_s"], "offered_requests_per_s": open70["offered_requests_per_s"],
            "load_fraction_of_capacity": 0.7, "load_sweep": loads,
            "capacity_keys_per_s": round(cap_keys_s, 1), "capacity_p99_ms": round(cap["p99_us"] / 1e3, 4),
            "plain_keys_per_s": round(plain_keys_s, 1), "served_vs_plain_speedup": round(cap_keys_s / plain_keys_s, 2),
            "uploads_during_run": open70["uploads_during_run"], "mean_keys_per_request": round(mean_keys, 1),
            "answers_equal_alone": exact, "budget_1GB": {"admitted": admitted, "rejected": tst["rejected_uploads"]},
            "budget_40GB_admitted": n_sk, "build_s": round(build_s, 1)}


if __name__ == "__main__":
    sys.exit(main())
