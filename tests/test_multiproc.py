"""Multi-process (world size 2, gloo on CPU) checks of the batched form's sharding: every rank
derives the same assignment on its own, the shards cover the batch exactly once, the loads are
balanced, and the max-over-ranks timing reduction the benchmark uses works across processes."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2406_04008_gb300 import sharding
from paper_2406_04008_gb300 import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    # the 64-collage batch's sizes (grid, element count) without building the outlines
    out = []
    for i in range(64):
        rng = W.PCG32(4000 + i)
        n = rng.randint(20, 800)
        grid = (256, 512, 1024)[rng.randint(0, 2)]
        out.append({"kind": [0] * n, "grid": grid})
    return out


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    probs = _batch()
    mine = sharding.shard(probs, world, rank)
    # gather every rank's shard (padded) and its load
    t = torch.full((64,), -1, dtype=torch.int64)
    t[: len(mine)] = torch.tensor(mine, dtype=torch.int64)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t)
    load = torch.tensor([sum(sharding.work_estimate(probs[i]) for i in mine)], dtype=torch.float64)
    loads = [torch.empty_like(load) for _ in range(world)]
    dist.all_gather(loads, load)
    # the benchmark's timing: the slowest rank's time
    mx = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put(([p[p >= 0].tolist() for p in parts], [float(x.item()) for x in loads],
               float(mx.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_sharding_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts, loads, mx = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(parts[0] + parts[1])
    assert flat == list(range(64))                    # exactly once
    assert set(parts[0]).isdisjoint(parts[1])
    assert parts == [sharding.shard(_batch(), 2, r) for r in range(2)]  # same without talking
    assert max(loads) / min(loads) < 1.05              # balanced
    assert mx == 2.0


@pytest.mark.parametrize("world", [1, 3, 8])
def test_lpt_assignment_properties(world):
    probs = _batch()
    owner, loads = sharding.assign([sharding.work_estimate(p) for p in probs], world)
    assert sorted(set(owner)) == list(range(min(world, len(probs))))
    heaviest = max(sharding.work_estimate(p) for p in probs)
    # LPT bound: no rank exceeds the average by more than one item
    assert max(loads) <= sum(loads) / world + heaviest
