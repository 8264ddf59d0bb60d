"""A CPU stand-in for a slab solver context (test infrastructure): the stage-level methods
SlabGroup drives (step_stage, step_stage_vjp, rows_pack, rows_unpack, max_dt), computed with
torch on the CPU for a toy nonlinear update whose stencil reaches 3 rows and 3 columns, like
a WENO5 stage.  It checks the decomposition logic (windows, exchange, its transpose, the
stage-wise reverse order, the CFL minimum, parameter-gradient sums) without a GPU.

Toy stage:  X = U_in with 3 ghost rows per y side (periodic wrap for a whole periodic grid,
else a copy of the edge row, as the library fills sides that border another slab),
    L(X)_j = theta * sum_{d=-3..3} c_d * g(X_{j+d}) + 0.1 * (roll_x(X, 1) - roll_x(X, -1)) ** 2 / 4,
    g(x) = x * |x| / (1 + x^2),
    U_out = a_k U_n + b_k (X + dt L(X)),
and max_dt = cfl / (1 + max |U|) over the window.  p_bar[0] collects d/d theta."""
import torch

RK_A = (0.0, 0.75, 1.0 / 3.0)
RK_B = (1.0, 0.25, 2.0 / 3.0)
C = (0.05, -0.2, 0.7, -1.0, 0.6, -0.15, 0.02)


class ToySlab:
    def __init__(self, plan, rank, theta=1.3):
        self.plan, self.rank = plan, rank
        lo, rows, own = plan.window(rank)
        self.window = (lo, rows, own, plan.nrows[rank])
        self.whole = plan.world == 1
        self.theta = theta
        self._acc = None
        self._next = 2

    def _pad(self, X):
        if self.whole and self.plan.periodic:
            return torch.cat([X[:, -3:], X, X[:, :3]], dim=1)
        return torch.cat([X[:, :1].expand(-1, 3, -1), X, X[:, -1:].expand(-1, 3, -1)], dim=1)

    def _L(self, X, theta):
        P = self._pad(X)
        g = P * P.abs() / (1.0 + P * P)
        rows = X.shape[1]
        out = torch.zeros_like(X)
        for d in range(7):
            out = out + C[d] * g[:, d:d + rows]
        mix = (torch.roll(X, 1, dims=2) - torch.roll(X, -1, dims=2)) ** 2 / 4.0
        return theta * out + 0.1 * mix

    def _stage(self, U_n, X, dt, k, theta):
        Y = X + dt * self._L(X, theta)
        return RK_B[k] * Y if k == 0 else RK_A[k] * U_n + RK_B[k] * Y

    def step_stage(self, U_n, U_in, U_out, dt, k):
        U_out.copy_(self._stage(U_n, U_in, dt, k, self.theta))
        return U_out

    def step_stage_vjp(self, U_in, dt, k, lam_out, lam_in, p_bar=None):
        assert k == 2 or k == self._next
        X = U_in.detach().clone().requires_grad_(True)
        Un = U_in.detach().clone().requires_grad_(True)  # only a_k * U_n, linear: value unused
        th = torch.tensor(self.theta, dtype=torch.float64, requires_grad=True)
        Y = self._stage(Un, X, dt, k, th)
        gX, gUn, gth = torch.autograd.grad(Y, (X, Un, th), lam_out, allow_unused=True)
        if k == 2:
            self._acc = torch.zeros_like(lam_out)
        if gUn is not None:
            self._acc = self._acc + gUn
        res = gX + self._acc if k == 0 else gX
        lam_in.copy_(res)
        if p_bar is not None:
            p_bar[0] += gth
        self._next = 2 if k == 0 else k - 1
        return lam_in

    def rows_pack(self, U, row0, nrows, buf, zero=False):
        flat = buf.view(-1)[:4 * nrows * U.shape[2]].view(4, nrows, U.shape[2])
        flat.copy_(U[:, row0:row0 + nrows])
        if zero:
            U[:, row0:row0 + nrows] = 0.0
        return buf

    def rows_unpack(self, U, row0, nrows, buf, add=False):
        src = buf.reshape(-1)[:4 * nrows * U.shape[2]].view(4, nrows, U.shape[2])
        if add:
            U[:, row0:row0 + nrows] += src
        else:
            U[:, row0:row0 + nrows] = src
        return U

    def max_dt(self, U, cfl):
        return cfl / (1.0 + float(U.abs().max()))
