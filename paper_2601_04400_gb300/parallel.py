"""Multi-GPU layouts (one process per GPU).

Batched path: independent instances are sharded over ranks with no exchange on the data path
(weak scaling).  shard(cells, world, rank) assigns instances greedily (largest first, to the
least loaded rank; ties to the lower rank), which keeps the per-rank cell counts within one
instance of each other and is the same on every rank without communication.

Single grid: decomposed into y slabs of whole rows (SlabPlan), one solver context per slab
(js_create_slab) holding `overlap` rows of each neighbour.  A stage output reads cells within
3 rows, so exchanging the overlap rows after every SSP-RK3 stage keeps every slab's owned rows
identical to the undecomposed grid (SlabGroup.step); the CFL step is the minimum over slabs.
The reverse step transposes each exchange: the adjoint of the overlap rows is added to the
owner's rows and cleared (SlabGroup.step_vjp); parameter gradients are summed over slabs.
The exchange moves contiguous [4, overlap, nx] row blocks, packed and unpacked by the
library's kernels, point to point between neighbours (torch.distributed P2P: NCCL between
GPUs, gloo between CPU processes), or by reference between slabs held by one process.
"""
import numpy as np

DOWN, UP = 0, 1  # message tags: rows sent to the lower / to the upper neighbour


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


# ---------------------------------------------------------------------------------------
# y-slab decomposition of one grid
# ---------------------------------------------------------------------------------------
def _takes_internals(slab):
    """Whether a slab solver can store stage internals (binding.Solver on a 2D grid)."""
    import inspect
    try:
        return "internals" in inspect.signature(slab.step_stage).parameters and slab.ny > 1
    except (TypeError, ValueError, AttributeError):
        return False


class SlabPlan:
    """Rows of an ny-row grid split over `world` slabs (sizes within one row of each other,
    lower ranks first), each slab holding `overlap` rows of each neighbour; with periodic y
    sides the first and last slabs are neighbours."""

    def __init__(self, ny, world, overlap=3, periodic=False):
        if world < 1 or ny < world:
            raise ValueError("need 1 <= world <= ny")
        self.ny, self.world, self.periodic = int(ny), int(world), bool(periodic)
        self.overlap = int(overlap) if world > 1 else 0
        base, rem = divmod(self.ny, self.world)
        self.nrows = [base + (1 if r < rem else 0) for r in range(self.world)]
        self.row0 = [sum(self.nrows[:r]) for r in range(self.world)]
        if self.world > 1:
            if self.overlap < 3:
                raise ValueError("overlap must be >= 3 rows (the stencil reach of a stage)")
            if min(self.nrows) < self.overlap:
                raise ValueError("every slab must own at least `overlap` rows")
            if self.periodic and max(self.nrows) + 2 * self.overlap > self.ny:
                raise ValueError("a periodic slab window would wrap onto itself")

    def lower(self, r):
        if r > 0:
            return r - 1
        return self.world - 1 if (self.periodic and self.world > 1) else None

    def upper(self, r):
        if r < self.world - 1:
            return r + 1
        return 0 if (self.periodic and self.world > 1) else None

    def window(self, r):
        """(first grid row, rows, local index of the first owned row) of slab r's window."""
        n, ov = self.nrows[r], self.overlap
        if self.world == 1:
            return 0, self.ny, 0
        if self.periodic:
            return (self.row0[r] - ov) % self.ny, n + 2 * ov, ov
        lo = max(0, self.row0[r] - ov)
        hi = min(self.ny, self.row0[r] + n + ov)
        return lo, hi - lo, self.row0[r] - lo

    def window_rows(self, r):
        lo, rows, _ = self.window(r)
        return (lo + np.arange(rows)) % self.ny

    def sends(self, r):
        """Forward exchange: (peer, tag, local first row, rows) of the blocks slab r sends."""
        _, _, own = self.window(r)
        n, ov, out = self.nrows[r], self.overlap, []
        if self.lower(r) is not None:
            out.append((self.lower(r), DOWN, own, ov))  # my lowest owned rows -> its upper overlap
        if self.upper(r) is not None:
            out.append((self.upper(r), UP, own + n - ov, ov))
        return out

    def recvs(self, r):
        """Forward exchange: (peer, tag, local first row, rows) of the blocks slab r receives."""
        _, _, own = self.window(r)
        n, ov, out = self.nrows[r], self.overlap, []
        if self.lower(r) is not None:
            out.append((self.lower(r), UP, own - ov, ov))
        if self.upper(r) is not None:
            out.append((self.upper(r), DOWN, own + n, ov))
        return out


class LocalTransport:
    """Every slab in this process: a message is handed over by reference."""

    def exchange(self, outgoing, incoming):
        """outgoing: {(src, dst, tag): buffer}; incoming: [(src, dst, tag, shape, like)];
        returns {(src, dst, tag): buffer} for the incoming messages."""
        return {(s, d, t): outgoing[(s, d, t)] for (s, d, t, _, _) in incoming}

    def min(self, x):
        return x

    def sum_(self, t):
        return t


class DistTransport:
    """Slabs in other processes reached through torch.distributed point-to-point messages
    (NCCL for CUDA buffers; gloo through host copies).  Messages between one pair of ranks are
    posted in tag order on both sides, so that backends that match by order pair them."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group)
        self.host = dist.get_backend(group) == "gloo"

    def _dev(self, t):
        return t.cpu() if self.host else t

    def exchange(self, outgoing, incoming):
        import torch
        d = self.dist
        ops, got, back = [], {}, []
        for (s, dst, tag), buf in sorted(outgoing.items(), key=lambda kv: (kv[0][1], kv[0][2])):
            ops.append(d.P2POp(d.isend, self._dev(buf).contiguous(), dst, self.group, tag))
        for (src, dst, tag, shape, like) in sorted(incoming, key=lambda m: (m[0], m[2])):
            b = torch.empty(shape, dtype=like.dtype, device="cpu" if self.host else like.device)
            ops.append(d.P2POp(d.irecv, b, src, self.group, tag))
            got[(src, dst, tag)] = b
            back.append(((src, dst, tag), like.device))
        if ops:
            for req in d.batch_isend_irecv(ops):
                req.wait()
        for key, dev in back:
            got[key] = got[key].to(dev)
        return got

    def min(self, x):
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64,
                         device="cpu" if self.host else torch.device("cuda", torch.cuda.current_device()))
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN, group=self.group)
        return float(t.item())

    def sum_(self, t):
        u = self._dev(t).clone()
        self.dist.all_reduce(u, group=self.group)
        return u.to(t.device)


class SlabGroup:
    """The slabs of a y-decomposed grid held by this process (`slabs`: {rank: solver}, solvers
    from binding.Solver.slab or any object with the same stage-level methods), exchanging
    halos with the other slabs through `transport` (LocalTransport when this process holds
    every slab, DistTransport with one slab per process).  States are {rank: [4, rows, nx]}
    arrays over each slab's window."""

    def __init__(self, plan, slabs, transport=None):
        self.plan, self.slabs = plan, dict(slabs)
        self.transport = transport if transport is not None else LocalTransport()
        for r, s in self.slabs.items():
            lo, rows, own = plan.window(r)
            info = getattr(s, "window", None)
            if info is not None and tuple(info) != (lo, rows, own, plan.nrows[r]):
                raise ValueError("slab %d window %s differs from the plan's %s" % (r, info, (lo, rows, own)))
        self._scratch = {}

    @classmethod
    def build(cls, prob, plan, ranks, transport=None, stream=None):
        """Slab solver contexts (js_create_slab) for `ranks` of the plan."""
        from .binding import Solver
        slabs = {r: Solver.slab(prob, plan.row0[r], plan.nrows[r], plan.overlap, stream) for r in ranks}
        return cls(plan, slabs, transport)

    # -- data placement ---------------------------------------------------------------
    def scatter(self, U):
        """{rank: window of U} for the slabs held here (U: [4, ny, nx] of the whole grid)."""
        import torch
        out = {}
        for r in self.slabs:
            idx = torch.as_tensor(self.plan.window_rows(r), device=U.device)
            out[r] = U.index_select(1, idx).contiguous()
        return out

    def gather(self, X, out=None):
        """Owned rows of the slabs held here, written into `out` ([4, ny, nx]) at their grid rows."""
        import torch
        if out is None:
            any_x = next(iter(X.values()))
            out = torch.zeros((any_x.shape[0], self.plan.ny, any_x.shape[2]), dtype=any_x.dtype, device=any_x.device)
        for r, x in X.items():
            _, _, own = self.plan.window(r)
            n = self.plan.nrows[r]
            out[:, self.plan.row0[r]:self.plan.row0[r] + n] = x[:, own:own + n]
        return out

    def _buf(self, key, like):
        b = self._scratch.get(key)
        if b is None or b.shape != like.shape or b.device != like.device:
            import torch
            b = torch.empty_like(like)
            self._scratch[key] = b
        return b

    # -- halo exchange ----------------------------------------------------------------
    def exchange(self, X, transpose=False):
        """Forward: overwrite every slab's overlap rows with the owners' rows.  transpose:
        add every slab's overlap rows into the owners' rows and clear them (the adjoint)."""
        import torch
        p = self.plan
        outgoing, incoming, land = {}, [], []
        for r, x in X.items():
            s = self.slabs[r]
            nx = x.shape[2]
            src = p.recvs(r) if transpose else p.sends(r)
            dst = p.sends(r) if transpose else p.recvs(r)
            for peer, tag, row, n in src:
                buf = torch.empty((4, n, nx), dtype=x.dtype, device=x.device)
                s.rows_pack(x, row, n, buf, zero=transpose)
                outgoing[(r, peer, tag)] = buf
            for peer, tag, row, n in dst:
                incoming.append((peer, r, tag, (4, n, nx), x))
                land.append((r, peer, tag, row, n))
        got = self.transport.exchange(outgoing, incoming)
        for r, peer, tag, row, n in land:
            self.slabs[r].rows_unpack(X[r], row, n, got[(peer, r, tag)], add=transpose)
        return X

    # -- forward ----------------------------------------------------------------------
    def max_dt(self, U, cfl):
        """The grid's CFL step: the minimum of the slabs' steps over every rank."""
        return self.transport.min(min(self.slabs[r].max_dt(U[r], cfl) for r in U))

    def step(self, U, dt, n_steps=1):
        """Advance every held slab's window in place by n_steps SSP-RK3 steps of size dt,
        exchanging halos after every stage."""
        for _ in range(int(n_steps)):
            X1 = {r: self._buf(("x1", r), u) for r, u in U.items()}
            X2 = {r: self._buf(("x2", r), u) for r, u in U.items()}
            for r, u in U.items():
                self.slabs[r].step_stage(u, u, X1[r], dt, 0)
            self.exchange(X1)
            for r, u in U.items():
                self.slabs[r].step_stage(u, X1[r], X2[r], dt, 1)
            self.exchange(X2)
            for r, u in U.items():
                self.slabs[r].step_stage(u, X2[r], u, dt, 2)
            self.exchange(U)
        return U

    def _stage(self, r, U_n, U_in, U_out, dt, k, internals):
        if internals:
            self.slabs[r].step_stage(U_n, U_in, U_out, dt, k, internals=True)
        else:
            self.slabs[r].step_stage(U_n, U_in, U_out, dt, k)

    # -- reverse ----------------------------------------------------------------------
    def step_vjp(self, U_n, dt, lam, p_bar=None):
        """Reverse of one step from U_n: returns ({rank: lam_n}, p_bar) where lam holds the
        adjoint of the step result on each slab's owned rows (its overlap rows are ignored)
        and p_bar (JS_NPARAM, accumulated into when given) is summed over all ranks."""
        import torch
        from .binding import JS_NPARAM
        X1 = {r: self._buf(("x1", r), u) for r, u in U_n.items()}
        X2 = {r: self._buf(("x2", r), u) for r, u in U_n.items()}
        # the recomputed stages 0 and 1 store their WENO5 internals for their reverse
        keep = {r: _takes_internals(s) for r, s in self.slabs.items()}
        for r, u in U_n.items():
            self._stage(r, u, u, X1[r], dt, 0, keep[r])
        self.exchange(X1)
        for r, u in U_n.items():
            self._stage(r, u, X1[r], X2[r], dt, 1, keep[r])
        self.exchange(X2)
        any_u = next(iter(U_n.values()))
        pb = torch.zeros(JS_NPARAM, dtype=torch.float64, device=any_u.device)
        L = {}
        for r, l in lam.items():
            L[r] = l.clone()
            _, rows, own = self.plan.window(r)
            n = self.plan.nrows[r]
            scratch = self._buf(("ov", r), L[r])
            self.slabs[r].rows_pack(L[r], 0, own, scratch, zero=True)  # clear the overlap rows
            self.slabs[r].rows_pack(L[r], own + n, rows - own - n, scratch, zero=True)
        Xs = (U_n, X1, X2)
        for k in (2, 1, 0):
            for r in L:
                if keep[r] and k < 2:
                    self.slabs[r].step_stage_vjp(Xs[k][r], dt, k, L[r], L[r], pb, internals=True)
                else:
                    self.slabs[r].step_stage_vjp(Xs[k][r], dt, k, L[r], L[r], pb)
            self.exchange(L, transpose=True)
        pb = self.transport.sum_(pb)
        if p_bar is not None:
            p_bar += pb
            pb = p_bar
        return L, pb
