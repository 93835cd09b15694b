"""The batched form sharded over ranks by whole collages (the benchmark's multi-GPU path): two
processes each step their share (sharding.shard, LPT, computed by every rank alone) in one batched
handle; gathered over gloo, every collage's loss terms, params and Adam state equal those of the
whole batch stepped in one process, bit for bit (deterministic mode).  Both processes use the one
GPU; neither waits on the other's kernels, only on the gloo gather of host tensors."""
import os
import socket

import numpy as np
import pytest
import torch

from paper_2406_04008_gb300 import sharding
from paper_2406_04008_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEPS = 4


def _problems():
    return [W.config_problem(4, i, n_elems=30 + 15 * i, grid=(256, 128, 192)[i % 3]) for i in range(6)]


def _kw():
    return dict(deterministic=1, n_levels=1, level_res=[1], level_iters=[10], use_graphs=1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_2406_04008_gb300 import build
    build.build()
    from paper_2406_04008_gb300.collage import Collage
    probs = _problems()
    mine = sharding.shard(probs, world, rank)
    col = Collage([probs[i] for i in mine], **_kw())
    col.step(STEPS)
    state, step, _ = col.get_state()
    out = {"idx": mine, "loss": col.loss().cpu().numpy(), "state": state.cpu().numpy(), "step": step,
           "n": [len(probs[i]["kind"]) for i in mine]}
    col.close()
    got = [None] * world
    dist.all_gather_object(got, out)
    if rank == 0:
        q.put(got)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_batch_equals_whole_batch():
    import torch.multiprocessing as mp
    from paper_2406_04008_gb300 import build
    build.build()
    from paper_2406_04008_gb300.collage import Collage
    probs = _problems()
    whole = Collage(probs, **_kw())
    whole.step(STEPS)
    wstate, wstep, _ = whole.get_state()
    wloss = whole.loss().cpu().numpy()
    wstate = wstate.cpu().numpy()
    whole.close()
    n = [len(p["kind"]) for p in probs]
    base = np.concatenate([[0], np.cumsum(n)])
    N = base[-1]

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    seen = []
    for part in got:
        assert part["step"] == wstep == STEPS
        off = 0
        S = sum(part["n"])
        for j, i in enumerate(part["idx"]):
            seen.append(i)
            assert np.array_equal(part["loss"][j], wloss[i]), i
            for blk in range(3):  # params, Adam m, Adam v
                a = part["state"][4 * (blk * S + off):4 * (blk * S + off + n[i])]
                b = wstate[4 * (blk * N + base[i]):4 * (blk * N + base[i] + n[i])]
                assert np.array_equal(a, b), (i, blk)
            off += n[i]
    assert sorted(seen) == list(range(len(probs)))
