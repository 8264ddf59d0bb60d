"""Multi-GPU layout of the batched path: independent instances are sharded over ranks with
no exchange on the data path (one process per GPU, weak scaling).  A single grid is not
decomposed: several GPUs run independent replicas of it.

shard(cells, world, rank) assigns instances greedily (largest first, to the least loaded
rank; ties to the lower rank), which keeps the per-rank cell counts within one instance of
each other and is the same on every rank without communication.
"""


def shard(cells, world, rank):
    """Indices of the instances (given their cell counts) that `rank` of `world` advances."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    load = [0] * world
    owner = [0] * len(cells)
    for k in sorted(range(len(cells)), key=lambda i: (-cells[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[k] = r
        load[r] += cells[k]
    return [k for k in range(len(cells)) if owner[k] == rank]


def rank_loads(cells, world):
    return [sum(cells[k] for k in shard(cells, world, r)) for r in range(world)]
