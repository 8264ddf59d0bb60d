"""Sharding of the batched path over ranks (host logic, CPU only): every instance is owned by
exactly one rank, loads are balanced, and world-size-2 gloo ranks that each compute their own
shard agree on the partition and on the total cells without exchanging instances."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2601_04400_gb300 import parallel
from paper_2601_04400_gb300 import workloads as W


def _cells():
    return [p.cells for p in W.batched_cases(64, seed=0)]


def test_shards_cover_every_instance_once():
    cells = _cells()
    for world in (1, 2, 3, 4, 8):
        owned = sorted(k for r in range(world) for k in parallel.shard(cells, world, r))
        assert owned == list(range(len(cells)))
        loads = parallel.rank_loads(cells, world)
        assert max(loads) - min(loads) <= max(cells)


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cells = _cells()
    mine = parallel.shard(cells, world, rank)
    t = torch.tensor([float(sum(cells[k] for k in mine)), float(len(mine))], dtype=torch.float64)
    dist.all_reduce(t)
    ids = torch.zeros(len(cells), dtype=torch.float64)
    ids[mine] = 1.0
    dist.all_reduce(ids)
    q.put((rank, t.tolist(), ids.tolist()))
    dist.destroy_process_group()


def test_gloo_ranks_agree_on_the_partition():
    world = 2
    port = 29500 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cells = _cells()
    for _, tot, ids in res:
        assert tot[0] == float(sum(cells)) and tot[1] == float(len(cells))
        assert all(v == 1.0 for v in ids)
