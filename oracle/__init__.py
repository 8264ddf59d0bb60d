"""FP64 CPU oracle for the JAX-Shock right-hand side and SSP-RK3 step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the CUDA library in
``paper_2601_04400_gb300`` and never imports it.

Problems are passed as any object with the attributes ``nx, ny, x0, y0, dx, dy, bc, wall,
gamma, mu, Pr, nu, inflow`` and ``sdf`` (see ``paper_2601_04400_gb300.workloads.Problem``).
Arrays are float64, conserved variables stacked as ``[4, ny, nx]`` (rho, rho u, rho v, E).
The parameter vector ``theta`` has 20 entries: gamma, mu, Pr, nu, then the inflow state
(rho, u, v, p) of the x-low, x-high, y-low and y-high sides.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OrGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("y0", C.c_double),
                ("dx", C.c_double), ("dy", C.c_double), ("bc", C.c_int * 4), ("wall", C.c_int),
                ("hllc_literal", C.c_int)]


_D = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_prim_to_cons.argtypes = [C.POINTER(OrGrid), _D, _D, _D]
        L.or_cons_to_prim.argtypes = [C.POINTER(OrGrid), _D, _D, _D]
        L.or_rhs.argtypes = [C.POINTER(OrGrid), _D, _D, _D, _D]
        L.or_step.argtypes = [C.POINTER(OrGrid), _D, _D, _D, _D, C.c_int]
        L.or_max_dt.argtypes = [C.POINTER(OrGrid), _D, _D, _D, C.c_double, _D]
        L.or_run_to.argtypes = [C.POINTER(OrGrid), _D, _D, _D, C.c_double, C.c_double, C.c_int, _D,
                                C.POINTER(C.c_int)]
        L.or_rhs_tangent.argtypes = [C.POINTER(OrGrid), _D, _D, _D, _D, _D, _D, _D]
        L.or_step_tangent.argtypes = [C.POINTER(OrGrid), _D, _D, _D, _D, _D, _D, C.c_int]
        L.or_count_rhs.argtypes = [C.POINTER(OrGrid), _D, _D, _D, C.POINTER(C.c_longlong)]
        L.or_ib_tables.argtypes = [C.POINTER(OrGrid), _D, C.POINTER(C.c_ubyte), C.POINTER(C.c_int),
                                   C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), _D, _D]
        L.or_weno5.argtypes = [_D, C.c_int, _D]
        L.or_weno5_beta.argtypes = [_D, _D]
        L.or_hllc.argtypes = [_D, _D, C.c_double, C.c_int, _D, _D]
        L.or_exact_riemann.argtypes = [C.c_double] * 9 + [_D, C.c_int, _D, _D, _D, _D]
        L.or_nn_set.argtypes = [_D, _D, _D]
        L.or_nn_eval.argtypes = [_D, C.c_int, C.c_int, _D]
        L.or_nn_nparam.restype = C.c_int
        L.or_fallback_faces.restype = C.c_longlong
        L.or_ib_fill.argtypes = [C.POINTER(OrGrid), _D, _D, _D, _D]
        L.or_set_threads.argtypes = [C.c_int]
        L.or_get_threads.restype = C.c_int
        _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise OracleError("%s failed with code %d" % (what, rc))


def _p(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def grid_of(prob, hllc_literal=False):
    g = OrGrid()
    g.nx, g.ny = int(prob.nx), int(prob.ny)
    g.x0, g.y0, g.dx, g.dy = float(prob.x0), float(prob.y0), float(prob.dx), float(prob.dy)
    for k in range(4):
        g.bc[k] = int(prob.bc[k])
    g.wall = int(getattr(prob, "wall", 0))
    g.hllc_literal = 1 if hllc_literal else 0
    return g


def theta_of(prob):
    th = np.zeros(20)
    th[0], th[1], th[2], th[3] = prob.gamma, prob.mu, prob.Pr, prob.nu
    th[4:] = np.asarray(prob.inflow, dtype=np.float64).reshape(16)
    return th


def _sdf(prob):
    s = getattr(prob, "sdf", None)
    return None if s is None else _f64(s)


def set_threads(n):
    lib().or_set_threads(int(n))


def threads():
    return lib().or_get_threads()


def prim_to_cons(prob, W, theta=None):
    g = grid_of(prob)
    th = _f64(theta_of(prob) if theta is None else theta)
    W = _f64(W)
    U = np.empty_like(W)
    _check(lib().or_prim_to_cons(C.byref(g), _p(th), _p(W), _p(U)), "prim_to_cons")
    return U


def cons_to_prim(prob, U, theta=None):
    g = grid_of(prob)
    th = _f64(theta_of(prob) if theta is None else theta)
    U = _f64(U)
    W = np.empty_like(U)
    _check(lib().or_cons_to_prim(C.byref(g), _p(th), _p(U), _p(W)), "cons_to_prim")
    return W


def rhs(prob, U, theta=None, hllc_literal=False):
    g = grid_of(prob, hllc_literal)
    th = _f64(theta_of(prob) if theta is None else theta)
    U = _f64(U)
    out = np.empty_like(U)
    _check(lib().or_rhs(C.byref(g), _p(th), _p(_sdf(prob)), _p(U), _p(out)), "rhs")
    return out


def step(prob, U, dts, theta=None):
    """SSP-RK3 steps with the given dt sequence; returns the new state."""
    g = grid_of(prob)
    th = _f64(theta_of(prob) if theta is None else theta)
    U = _f64(U).copy()
    dts = _f64(np.atleast_1d(dts))
    _check(lib().or_step(C.byref(g), _p(th), _p(_sdf(prob)), _p(U), _p(dts), len(dts)), "step")
    return U


def max_dt(prob, U, cfl, theta=None):
    g = grid_of(prob)
    th = _f64(theta_of(prob) if theta is None else theta)
    U = _f64(U)
    dt = C.c_double(0.0)
    _check(lib().or_max_dt(C.byref(g), _p(th), _p(_sdf(prob)), _p(U), float(cfl), C.byref(dt)), "max_dt")
    return dt.value


def run_to(prob, U, cfl, t_end, max_steps=1000000, theta=None):
    """CFL-driven run to t_end (last step clipped).  Returns (U, dts)."""
    g = grid_of(prob)
    th = _f64(theta_of(prob) if theta is None else theta)
    U = _f64(U).copy()
    dts = np.zeros(max_steps)
    n = C.c_int(0)
    _check(lib().or_run_to(C.byref(g), _p(th), _p(_sdf(prob)), _p(U), float(cfl), float(t_end),
                           int(max_steps), _p(dts), C.byref(n)), "run_to")
    return U, dts[:n.value].copy()


def rhs_tangent(prob, U, dU, dtheta, theta=None):
    g = grid_of(prob)
    th = _f64(theta_of(prob) if theta is None else theta)
    U, dU, dth = _f64(U), _f64(dU), _f64(dtheta)
    L, dL = np.empty_like(U), np.empty_like(U)
    _check(lib().or_rhs_tangent(C.byref(g), _p(th), _p(dth), _p(_sdf(prob)), _p(U), _p(dU), _p(L), _p(dL)),
           "rhs_tangent")
    return L, dL


def step_tangent(prob, U, dU, dtheta, dts, theta=None):
    """Forward-mode derivative of len(dts) SSP-RK3 steps.  Returns (U, dU)."""
    g = grid_of(prob)
    th = _f64(theta_of(prob) if theta is None else theta)
    U, dU = _f64(U).copy(), _f64(dU).copy()
    dth = _f64(dtheta)
    dts = _f64(np.atleast_1d(dts))
    _check(lib().or_step_tangent(C.byref(g), _p(th), _p(dth), _p(_sdf(prob)), _p(U), _p(dU), _p(dts),
                                 len(dts)), "step_tangent")
    return U, dU


def count_rhs(prob, U, theta=None):
    """Operation tally of one RHS evaluation: dict(add, mul, div, sqrt, cmp)."""
    g = grid_of(prob)
    th = _f64(theta_of(prob) if theta is None else theta)
    out = (C.c_longlong * 5)()
    _check(lib().or_count_rhs(C.byref(g), _p(th), _p(_sdf(prob)), _p(_f64(U)), out), "count_rhs")
    return dict(zip(("add", "mul", "div", "sqrt", "cmp"), list(out)))


def ib_tables(prob):
    """Immersed-boundary classification and ghost interpolation tables."""
    g = grid_of(prob)
    sdf = _sdf(prob)
    n = prob.nx * prob.ny
    tag = np.zeros(n, dtype=np.uint8)
    ng = C.c_int(0)
    L = lib()
    _check(L.or_ib_tables(C.byref(g), _p(sdf), tag.ctypes.data_as(C.POINTER(C.c_ubyte)), C.byref(ng), 0,
                          None, None, None, None), "ib_tables")
    k = ng.value
    gcell = np.zeros(max(k, 1), dtype=np.int32)
    icell = np.zeros(max(4 * k, 1), dtype=np.int32)
    w = np.zeros(max(4 * k, 1))
    nrm = np.zeros(max(2 * k, 1))
    _check(L.or_ib_tables(C.byref(g), _p(sdf), tag.ctypes.data_as(C.POINTER(C.c_ubyte)), C.byref(ng), k,
                          gcell.ctypes.data_as(C.POINTER(C.c_int)), icell.ctypes.data_as(C.POINTER(C.c_int)),
                          _p(w), _p(nrm)), "ib_tables")
    return dict(tag=tag.reshape(prob.ny, prob.nx), gcell=gcell[:k], icell=icell[:4 * k].reshape(k, 4),
                w=w[:4 * k].reshape(k, 4), nrm=nrm[:2 * k].reshape(k, 2))


def fallback_faces():
    """Faces at which the positivity fallback (first-order cell states) was taken since the
    last call, over every RHS evaluation in between; resets the count."""
    return int(lib().or_fallback_faces())


def ib_fill(prob, U, theta=None):
    """The immersed-boundary ghost fill alone: U with every ghost cell set to its mirrored
    image-point state (other cells copied)."""
    g = grid_of(prob)
    th = _f64(theta_of(prob) if theta is None else theta)
    U = _f64(U)
    out = np.empty_like(U)
    _check(lib().or_ib_fill(C.byref(g), _p(th), _p(_sdf(prob)), _p(U), _p(out)), "ib_fill")
    return out


def weno5(q, linear=False):
    q = _f64(q)
    out = C.c_double(0.0)
    lib().or_weno5(_p(q), 1 if linear else 0, C.byref(out))
    return out.value


def weno5_beta(q):
    q = _f64(q)
    b = np.zeros(3)
    lib().or_weno5_beta(_p(q), _p(b))
    return b


def hllc(qL, qR, gamma, literal=False):
    """HLLC flux for states (rho, u_normal, u_tangential, p).  Returns (F, diag dict)."""
    qL, qR = _f64(qL), _f64(qR)
    F = np.zeros(4)
    d = np.zeros(27)
    lib().or_hllc(_p(qL), _p(qR), float(gamma), 1 if literal else 0, _p(F), _p(d))
    diag = dict(sL=d[0], sR=d[1], ss=d[2], UsL=d[3:7], UsR=d[7:11], UL=d[11:15], UR=d[15:19],
                FL=d[19:23], FR=d[23:27])
    return F, diag


def exact_riemann(left, right, gamma, x, x0, t):
    """Exact solution of the 1D Riemann problem; left/right = (rho, u, p)."""
    x = _f64(x)
    n = len(x)
    r, u, p, star = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(4)
    _check(lib().or_exact_riemann(float(left[0]), float(left[1]), float(left[2]), float(right[0]),
                                  float(right[1]), float(right[2]), float(gamma), float(x0), float(t),
                                  _p(x), n, _p(r), _p(u), _p(p), _p(star)), "exact_riemann")
    return r, u, p, dict(p=star[0], u=star[1], rhoL=star[2], rhoR=star[3])


# ---------------------------------------------------------------------------------------
# neural flux (Sec. 2.3)
# ---------------------------------------------------------------------------------------
def nn_nparam():
    return lib().or_nn_nparam()


def nn_set(w, norm, dw=None):
    """Switch the neural flux on for every later call: w = the network's parameters, norm =
    (mean[4], sd[4], scale[4]) of the frame channels (rho, normal momentum, tangential
    momentum, E); dw = tangent of w for the *_tangent calls.  nn_set(None, None) switches it
    off."""
    if w is None:
        _check(lib().or_nn_set(None, None, None), "nn_set")
        return
    w = _f64(w).reshape(-1)
    if w.size != nn_nparam():
        raise ValueError("expected %d network parameters" % nn_nparam())
    dw = None if dw is None else _f64(dw).reshape(-1)
    _check(lib().or_nn_set(_p(w), _p(dw), _p(_f64(norm).reshape(12))), "nn_set")


def nn_eval(X):
    """The network on one normalised image X[4, H, W] -> scaled flux Y[4, H, W]."""
    X = _f64(X)
    Y = np.empty_like(X)
    _check(lib().or_nn_eval(_p(X), X.shape[1], X.shape[2], _p(Y)), "nn_eval")
    return Y


class neural:
    """Context manager: the neural flux switched on inside the block."""

    def __init__(self, w, norm, dw=None):
        self.args = (w, norm, dw)

    def __enter__(self):
        nn_set(self.args[0], self.args[1], dw=self.args[2])
        return self

    def __exit__(self, *exc):
        nn_set(None, None)
        return False

