"""Independent sketches sharded across ranks with no data-path collective, exercised with
world_size-2 gloo process groups on the CPU (the oracle stands in for each rank's engine)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads as wl
from paper_1701_04148_gb300 import shard


def test_assign_covers_each_sketch_once_and_balances():
    plan = wl.many_sketch_plan(1024, seed=3)
    lengths = [p["n"] for p in plan]
    for world in (1, 2, 3, 8):
        owner = shard.assign(lengths, world)
        assert sorted(set(owner)) == list(range(world))
        assert sum(len(shard.owned(lengths, world, r)) for r in range(world)) == len(lengths)
        assert shard.imbalance(lengths, world) < 1.05
    assert shard.assign(lengths, 4) == shard.assign(lengths, 4)  # deterministic


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, plan, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lengths = [p["n"] for p in plan]
    mine = shard.owned(lengths, world, rank)
    digests = {}
    for i in mine:
        p = plan[i]
        st, _ = wl.mixed_stream(p["n"], p["distinct"], p["s"], 0.1, 4, seed=p["seed"])
        o = oracle.Sketch(4, p["w"], 16, 4, p["seed"])
        o.update(st.keys.numpy(), st.ops.numpy(), S=max(2, p["n"] // 8))
        digests[i] = int(np.uint64(o.A.astype(np.uint64).sum()) * np.uint64(1000003) + np.uint64(o.B.sum()))
    # host-side gather of results (bookkeeping only) and max-over-ranks of a timing value
    gathered = [None] * world
    dist.all_gather_object(gathered, digests)
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        merged = {}
        for g in gathered:
            merged.update(g)
        out_q.put((merged, float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_rank_results():
    plan = wl.many_sketch_plan(12, seed=21, w_log2=(6.0, 9.0), n_log10=(2.0, 3.5))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, plan, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged, tmax = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sorted(merged) == list(range(len(plan))) and tmax == 2.0
    for i, p in enumerate(plan):
        st, _ = wl.mixed_stream(p["n"], p["distinct"], p["s"], 0.1, 4, seed=p["seed"])
        o = oracle.Sketch(4, p["w"], 16, 4, p["seed"])
        o.update(st.keys.numpy(), st.ops.numpy(), S=max(2, p["n"] // 8))
        want = int(np.uint64(o.A.astype(np.uint64).sum()) * np.uint64(1000003) + np.uint64(o.B.sum()))
        assert merged[i] == want

