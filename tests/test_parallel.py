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


# ---------------------------------------------------------------------------------------
# y-slab decomposition of one grid (host logic with the CPU stand-in slab of slab_toy)
# ---------------------------------------------------------------------------------------
from slab_toy import ToySlab  # noqa: E402

PLANS = [(40, 2, 3, False), (40, 3, 4, False), (41, 4, 3, True), (30, 2, 5, True), (37, 5, 3, False),
         (24, 2, 12, False)]


@pytest.mark.parametrize("ny,world,ov,per", PLANS)
def test_slab_plan_messages_cover_the_overlaps(ny, world, ov, per):
    p = parallel.SlabPlan(ny, world, ov, per)
    assert sum(p.nrows) == ny and max(p.nrows) - min(p.nrows) <= 1
    for r in range(world):
        rows_r = p.window_rows(r)
        lo, n, own = p.window(r)
        assert list(rows_r[own:own + p.nrows[r]]) == list(range(p.row0[r], p.row0[r] + p.nrows[r]))
        for peer, tag, row, m in p.sends(r):
            match = [x for x in p.recvs(peer) if x[0] == r and x[1] == tag]
            assert len(match) == 1
            _, _, prow, pm = match[0]
            assert pm == m and own <= row and row + m <= own + p.nrows[r]
            assert list(rows_r[row:row + m]) == list(p.window_rows(peer)[prow:prow + m])
        got = sorted(i for _, _, row, m in p.recvs(r) for i in range(row, row + m))
        assert got == [i for i in range(n) if not own <= i < own + p.nrows[r]]


def test_slab_plan_rejects_bad_layouts():
    for args in [(40, 2, 2, False), (10, 4, 3, False), (20, 2, 6, True), (3, 4, 3, False)]:
        with pytest.raises(ValueError):
            parallel.SlabPlan(*args)


def _toy_state(ny, nx=12, seed=0):
    g = torch.Generator().manual_seed(seed)
    return torch.rand((4, ny, nx), generator=g, dtype=torch.float64) * 2.0 - 0.5


def _toy_group(ny, world, ov, per):
    plan = parallel.SlabPlan(ny, world, ov, per)
    return parallel.SlabGroup(plan, {r: ToySlab(plan, r) for r in range(world)})


def _toy_forward(G, U0, steps, cfl=0.4):
    U = G.scatter(U0)
    dts = []
    for _ in range(steps):
        dt = G.max_dt(U, cfl)
        dts.append(dt)
        G.step(U, dt, 1)
    return G.gather(U), dts


@pytest.mark.parametrize("ny,world,ov,per", PLANS)
def test_slab_group_forward_equals_whole_grid(ny, world, ov, per):
    U0 = _toy_state(ny)
    ref, dts_ref = _toy_forward(_toy_group(ny, 1, 3, per), U0, 4)
    out, dts = _toy_forward(_toy_group(ny, world, ov, per), U0, 4)
    assert dts == dts_ref
    assert torch.equal(out, ref)


@pytest.mark.parametrize("ny,world,ov,per", PLANS)
def test_slab_group_reverse_equals_whole_grid(ny, world, ov, per):
    U0 = _toy_state(ny, seed=1)
    lam = _toy_state(ny, seed=2)
    G1 = _toy_group(ny, 1, 3, per)
    l1, p1 = G1.step_vjp(G1.scatter(U0), 0.03, G1.scatter(lam))
    ref = G1.gather(l1)
    G = _toy_group(ny, world, ov, per)
    lw, pw = G.step_vjp(G.scatter(U0), 0.03, G.scatter(lam))
    out = G.gather(lw)
    assert (out - ref).abs().max() <= 1e-13 * ref.abs().max()
    assert abs(float(pw[0] - p1[0])) <= 1e-12 * abs(float(p1[0])) and float(p1[0]) != 0.0
    for r, l in lw.items():  # the overlap rows of the returned adjoint are cleared
        _, rows, own = G.plan.window(r)
        n = G.plan.nrows[r]
        assert float(l[:, :own].abs().sum()) == 0.0 and float(l[:, own + n:].abs().sum()) == 0.0


@pytest.mark.parametrize("ny,world,ov,per", PLANS[:4])
def test_exchange_transpose_is_its_adjoint(ny, world, ov, per):
    G = _toy_group(ny, world, ov, per)
    g = torch.Generator().manual_seed(5)
    x = {r: torch.randn((4, G.plan.window(r)[1], 7), generator=g, dtype=torch.float64) for r in range(world)}
    y = {r: torch.randn_like(v) for r, v in x.items()}
    Ex = G.exchange({r: v.clone() for r, v in x.items()})
    ETy = G.exchange({r: v.clone() for r, v in y.items()}, transpose=True)
    lhs = sum(float((Ex[r] * y[r]).sum()) for r in x)
    rhs = sum(float((x[r] * ETy[r]).sum()) for r in x)
    assert abs(lhs - rhs) <= 1e-12 * sum(float(v.abs().sum()) for v in y.values())


def _slab_worker(rank, world, port, ny, ov, per, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        plan = parallel.SlabPlan(ny, world, ov, per)
        G = parallel.SlabGroup(plan, {rank: ToySlab(plan, rank)}, parallel.DistTransport())
        out, dts = _toy_forward(G, _toy_state(ny), 3)
        lw, pw = G.step_vjp(G.scatter(_toy_state(ny, seed=1)), 0.03, G.scatter(_toy_state(ny, seed=2)))
        q.put((rank, out.numpy(), dts, G.gather(lw).numpy(), float(pw[0])))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ny,world,ov,per", [(40, 2, 4, False), (41, 3, 3, True), (30, 2, 5, True)])
def test_gloo_slab_ranks_equal_whole_grid(ny, world, ov, per):
    port = 29600 + (os.getpid() + 7 * world + ny) % 1000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_slab_worker, args=(r, world, port, ny, ov, per, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref, dts_ref = _toy_forward(_toy_group(ny, 1, 3, per), _toy_state(ny), 3)
    G1 = _toy_group(ny, 1, 3, per)
    l1, p1 = G1.step_vjp(G1.scatter(_toy_state(ny, seed=1)), 0.03, G1.scatter(_toy_state(ny, seed=2)))
    lref = G1.gather(l1)
    plan = parallel.SlabPlan(ny, world, ov, per)
    out = torch.zeros_like(ref)
    lam = torch.zeros_like(ref)
    for rank, o, dts, lw, pw in res:
        assert dts == dts_ref  # every rank takes the grid's CFL step
        rows = slice(plan.row0[rank], plan.row0[rank] + plan.nrows[rank])
        out[:, rows] = torch.from_numpy(o)[:, rows]
        lam[:, rows] = torch.from_numpy(lw)[:, rows]
        assert abs(pw - float(p1[0])) <= 1e-12 * abs(float(p1[0]))  # summed over the ranks
    assert torch.equal(out, ref)
    assert (lam - lref).abs().max() <= 1e-13 * lref.abs().max()
