"""Thin ctypes binding of libjaxshock.so (include/jaxshock.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels; PyTorch only provides device
memory and the stream.  Functions keep the C names (js_create, js_rhs, js_step, ...) and
take torch tensors: float64, CUDA, contiguous, conserved variables shaped [4, ny, nx].
The library is loaded on first use; if it is missing and cannot be built, loading raises --
there is no CPU fallback.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

JS_OK, JS_ERR_ARG, JS_ERR_CUDA, JS_ERR_NONPHYSICAL, JS_ERR_TIMEOUT, JS_ERR_IB, JS_ERR_NOMEM = 0, -1, -2, -3, -4, -5, -6
JS_ARITH_FAST, JS_ARITH_IEEE = 0, 1
JS_NPARAM = 20
JS_TAPE_WENO = 1
JS_STAGE_INTERNALS = 16
JS_NN_NPARAM = 6388
JS_NN_F64, JS_NN_F32, JS_NN_BF16 = 0, 1, 2
JS_NN_LAYERWISE = 0x100

_lib = None


class JsGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("y0", C.c_double),
                ("dx", C.c_double), ("dy", C.c_double)]


class JsBoundary(C.Structure):
    _fields_ = [("kind", C.c_int * 4), ("inflow", (C.c_double * 4) * 4)]


class JsParams(C.Structure):
    _fields_ = [("gamma", C.c_double), ("mu", C.c_double), ("Pr", C.c_double), ("nu", C.c_double),
                ("wall", C.c_int)]


class JsError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s: %s (%d)" % (what, strerror(code), code))
        self.code = code


_P = C.c_void_p
_D = C.c_double
_I = C.c_int

# name -> (restype, argtypes)
SIGNATURES = {
    "js_create": (_I, [C.POINTER(JsGrid), C.POINTER(JsParams), C.POINTER(JsBoundary), _P, _P, C.POINTER(_P)]),
    "js_destroy": (None, [_P]),
    "js_set_params": (_I, [_P, C.POINTER(JsParams), C.POINTER(JsBoundary)]),
    "js_set_stream": (_I, [_P, _P]),
    "js_prim_to_cons": (_I, [_P, _P, _P]),
    "js_rhs": (_I, [_P, _P, _P]),
    "js_max_dt": (_I, [_P, _P, _D, C.POINTER(_D)]),
    "js_step": (_I, [_P, _P, _D, _I]),
    "js_step_cfl": (_I, [_P, _P, _D, _I, _P, _D, _P]),
    "js_rhs_vjp": (_I, [_P, _P, _P, _P, _P]),
    "js_step_vjp": (_I, [_P, _P, _D, _P, _P, _P]),
    "js_sync_status": (_I, [_P]),
    "js_ib_info": (_I, [_P, C.POINTER(_I), _P]),
    "js_tape_reserve": (_I, [_P, _I]),
    "js_tape_reserve_ex": (_I, [_P, _I, _I]),
    "js_set_neural": (_I, [_P, _P, _P, _P, _I]),
    "js_block_average": (_I, [_P, _I, _I, _I, _I, _P, _P]),
    "js_nn_eval": (_I, [_P, _P, _I, _I, _P]),
    "js_nn_eval_vjp": (_I, [_P, _P, _I, _I, _P, _P]),
    "js_step_taped": (_I, [_P, _P, _D, _I]),
    "js_step_stage": (_I, [_P, _P, _P, _P, _D, _I]),
    "js_step_stage_vjp": (_I, [_P, _P, _D, _I, _P, _P, _P]),
    "js_create_slab": (_I, [C.POINTER(JsGrid), C.POINTER(JsParams), C.POINTER(JsBoundary), _P, _I, _I, _I, _P,
                            C.POINTER(_P)]),
    "js_slab_info": (_I, [_P, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    "js_rows_pack": (_I, [_P, _P, _I, _I, _P, _I]),
    "js_rows_unpack": (_I, [_P, _P, _I, _I, _P, _I]),
    "js_step_vjp_taped": (_I, [_P, _I, _D, _P, _P, _P]),
    "js_set_arith": (_I, [_P, _I]),
    "js_get_arith": (_I, [_P, C.POINTER(_I)]),
    "js_set_tuning": (_I, [_P, _I]),
    "js_get_tuning": (_I, [_P, C.POINTER(_I), C.POINTER(_I)]),
    "js_profile_begin": (_I, [_P, _I]),
    "js_profile_end": (_I, [_P, C.POINTER(_D), C.POINTER(_I), C.POINTER(C.c_longlong)]),
    "js_max_dt_noalloc": (_I, [C.POINTER(JsGrid), C.POINTER(JsParams), _P, _P, _D, _P, C.POINTER(_D)]),
    "js_strerror": (C.c_char_p, [_I]),
    "js_batch_create": (_I, [_I, C.POINTER(JsGrid), C.POINTER(JsParams), C.POINTER(JsBoundary), C.POINTER(_P), _P,
                             C.POINTER(_P)]),
    "js_batch_set_states": (_I, [_P, C.POINTER(_P)]),
    "js_batch_step": (_I, [_P, _D, _I, _P, _P]),
    "js_batch_step_vjp": (_I, [_P, C.POINTER(_P), C.POINTER(_D), C.POINTER(_P), C.POINTER(_P), C.POINTER(_P)]),
    "js_batch_step_fixed": (_I, [_P, _I, _P]),
    "js_batch_set_tuning": (_I, [_P, _I, _I]),
    "js_batch_get_tuning": (_I, [_P, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    "js_batch_set_reverse_launch": (_I, [_P, _I]),
    "js_batch_get_reverse_launch": (_I, [_P, C.POINTER(_I)]),
    "js_batch_rollout_vjp": (_I, [_P, _I, _P, _I, C.POINTER(_P), C.POINTER(_P)]),
    "js_batch_rollout_forward": (_I, [_P, _D, _I, _I, _P]),
    "js_batch_rollout_spacing": (_I, [_P, _I, C.POINTER(_I)]),
    "js_batch_sync_status": (_I, [_P]),
    "js_batch_info": (_I, [_P, C.POINTER(_I), C.POINTER(_I), C.POINTER(C.c_longlong)]),
    "js_batch_instance": (_P, [_P, _I]),
    "js_batch_test_timeout": (_I, [_P, _D]),
    "js_batch_destroy": (None, [_P]),
}


def library_path():
    return _build.LIB


def lib():
    """Load libjaxshock.so (building it in-tree if it is absent)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            _build.build()
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(code):
    return lib().js_strerror(int(code)).decode()


def _check(rc, what):
    if rc != JS_OK:
        raise JsError(rc, what)


def _ptr(t):
    """Device pointer of a float64 CUDA tensor (must be contiguous)."""
    import torch
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream_ptr(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def make_structs(nx, ny, x0, y0, dx, dy, bc, gamma, mu, Pr, nu, inflow, wall=0):
    g = JsGrid(int(nx), int(ny), float(x0), float(y0), float(dx), float(dy))
    p = JsParams(float(gamma), float(mu), float(Pr), float(nu), int(wall))
    b = JsBoundary()
    inflow = np.asarray(inflow, dtype=np.float64).reshape(4, 4)
    for s in range(4):
        b.kind[s] = int(bc[s])
        for k in range(4):
            b.inflow[s][k] = float(inflow[s, k])
    return g, p, b


# ---------------------------------------------------------------------------------------
# C-named wrappers
# ---------------------------------------------------------------------------------------
def js_create(grid, params, boundary, sdf=None, stream=None):
    sdf_p = None
    if sdf is not None:
        sdf = np.ascontiguousarray(sdf, dtype=np.float64)
        sdf_p = sdf.ctypes.data_as(C.c_void_p)
    out = C.c_void_p()
    _check(lib().js_create(C.byref(grid), C.byref(params), C.byref(boundary), sdf_p, _stream_ptr(stream),
                           C.byref(out)), "js_create")
    return out


def js_create_slab(grid, params, boundary, sdf, row0, nrows, overlap, stream=None):
    sdf_p = None
    if sdf is not None:
        sdf = np.ascontiguousarray(sdf, dtype=np.float64)
        sdf_p = sdf.ctypes.data_as(C.c_void_p)
    out = C.c_void_p()
    _check(lib().js_create_slab(C.byref(grid), C.byref(params), C.byref(boundary), sdf_p, int(row0), int(nrows),
                                int(overlap), _stream_ptr(stream), C.byref(out)), "js_create_slab")
    return out


def js_slab_info(ctx):
    v = [C.c_int(0) for _ in range(4)]
    _check(lib().js_slab_info(ctx, *[C.byref(x) for x in v]), "js_slab_info")
    return tuple(x.value for x in v)


def js_destroy(ctx):
    lib().js_destroy(ctx)


def js_set_params(ctx, params, boundary):
    _check(lib().js_set_params(ctx, C.byref(params), C.byref(boundary)), "js_set_params")


def js_set_stream(ctx, stream=None):
    _check(lib().js_set_stream(ctx, _stream_ptr(stream)), "js_set_stream")


def js_prim_to_cons(ctx, W, U):
    _check(lib().js_prim_to_cons(ctx, _ptr(W), _ptr(U)), "js_prim_to_cons")


def js_rhs(ctx, U, dUdt):
    _check(lib().js_rhs(ctx, _ptr(U), _ptr(dUdt)), "js_rhs")


def js_max_dt(ctx, U, cfl):
    dt = C.c_double(0.0)
    _check(lib().js_max_dt(ctx, _ptr(U), float(cfl), C.byref(dt)), "js_max_dt")
    return dt.value


def js_step(ctx, U, dt, n_steps):
    _check(lib().js_step(ctx, _ptr(U), float(dt), int(n_steps)), "js_step")


def js_rhs_vjp(ctx, U, lam, U_bar, p_bar=None):
    _check(lib().js_rhs_vjp(ctx, _ptr(U), _ptr(lam), _ptr(U_bar), _ptr(p_bar)), "js_rhs_vjp")


def js_step_vjp(ctx, U_n, dt, lam_np1, lam_n, p_bar=None):
    _check(lib().js_step_vjp(ctx, _ptr(U_n), float(dt), _ptr(lam_np1), _ptr(lam_n), _ptr(p_bar)), "js_step_vjp")


def js_profile_begin(ctx, capacity):
    _check(lib().js_profile_begin(ctx, int(capacity)), "js_profile_begin")


def js_profile_end(ctx):
    """Returns (summed stage-kernel ms, stage launches timed, kernels launched)."""
    ms, n, k = C.c_double(0.0), C.c_int(0), C.c_longlong(0)
    _check(lib().js_profile_end(ctx, C.byref(ms), C.byref(n), C.byref(k)), "js_profile_end")
    return ms.value, n.value, k.value


def js_max_dt_noalloc(grid, params, U, tag=None, cfl=0.5, stream=None):
    """Context-free CFL step whose scratch is a static device array (no device allocation).
    tag: optional uint8 CUDA tensor [ny, nx] (0 = fluid)."""
    import torch
    tp = None
    if tag is not None:
        if not (tag.is_cuda and tag.dtype == torch.uint8 and tag.is_contiguous()):
            raise ValueError("tag must be a contiguous uint8 CUDA tensor")
        tp = C.c_void_p(tag.data_ptr())
    dt = C.c_double(0.0)
    _check(lib().js_max_dt_noalloc(C.byref(grid), C.byref(params), _ptr(U), tp, float(cfl), _stream_ptr(stream),
                                   C.byref(dt)), "js_max_dt_noalloc")
    return dt.value


def js_sync_status(ctx):
    return lib().js_sync_status(ctx)


def js_ib_info(ctx, nx, ny):
    n = C.c_int(0)
    tag = np.zeros((ny, nx), dtype=np.uint8)
    _check(lib().js_ib_info(ctx, C.byref(n), tag.ctypes.data_as(C.c_void_p)), "js_ib_info")
    return n.value, tag


# ---------------------------------------------------------------------------------------
# convenience object owning a context
# ---------------------------------------------------------------------------------------
class Solver:
    """One solver context: a grid, its parameters, boundaries and optional immersed body."""

    def __init__(self, nx, ny, x0, y0, dx, dy, bc=(0, 0, 0, 0), gamma=1.4, mu=0.0, Pr=0.72, nu=0.0,
                 inflow=None, wall=0, sdf=None, stream=None):
        if inflow is None:
            inflow = np.tile([1.0, 0.0, 0.0, 1.0], (4, 1))
        self.nx, self.ny = int(nx), int(ny)
        self.dx, self.dy = float(dx), float(dy)
        self._spec = dict(nx=nx, ny=ny, x0=x0, y0=y0, dx=dx, dy=dy, bc=tuple(bc), gamma=gamma, mu=mu, Pr=Pr,
                          nu=nu, inflow=np.asarray(inflow, dtype=np.float64).reshape(4, 4), wall=wall)
        self._g, self._p, self._b = make_structs(**self._spec)
        self.has_ib = sdf is not None
        self.ctx = js_create(self._g, self._p, self._b, sdf, stream)

    @classmethod
    def from_problem(cls, prob, stream=None):
        return cls(prob.nx, prob.ny, prob.x0, prob.y0, prob.dx, prob.dy, prob.bc, prob.gamma, prob.mu, prob.Pr,
                   prob.nu, prob.inflow, getattr(prob, "wall", 0), prob.sdf, stream)

    @classmethod
    def slab(cls, prob, row0, nrows, overlap, stream=None):
        """Context of the y slab owning rows [row0, row0 + nrows) of the problem's grid, holding
        `overlap` rows of each neighbour (js_create_slab).  Its arrays are [4, rows, nx] over
        the window; `window` = (first grid row, rows, local first owned row, owned rows)."""
        self = cls.__new__(cls)
        self._spec = dict(nx=prob.nx, ny=prob.ny, x0=prob.x0, y0=prob.y0, dx=prob.dx, dy=prob.dy, bc=tuple(prob.bc),
                          gamma=prob.gamma, mu=prob.mu, Pr=prob.Pr, nu=prob.nu,
                          inflow=np.asarray(prob.inflow, dtype=np.float64).reshape(4, 4),
                          wall=getattr(prob, "wall", 0))
        self._g, self._p, self._b = make_structs(**self._spec)
        self.has_ib = prob.sdf is not None
        self.ctx = js_create_slab(self._g, self._p, self._b, prob.sdf, row0, nrows, overlap, stream)
        self.window = js_slab_info(self.ctx)
        self.nx, self.ny = int(prob.nx), self.window[1]
        self.dx, self.dy = float(prob.dx), float(prob.dy)
        return self

    @property
    def shape(self):
        return (4, self.ny, self.nx)

    def set_params(self, gamma=None, mu=None, Pr=None, nu=None, inflow=None):
        for k, v in (("gamma", gamma), ("mu", mu), ("Pr", Pr), ("nu", nu)):
            if v is not None:
                self._spec[k] = float(v)
        if inflow is not None:
            self._spec["inflow"] = np.asarray(inflow, dtype=np.float64).reshape(4, 4)
        self._g, self._p, self._b = make_structs(**self._spec)
        js_set_params(self.ctx, self._p, self._b)

    def set_stream(self, stream=None):
        js_set_stream(self.ctx, stream)

    def set_neural(self, w, norm=None, w_bar=None, fp32=False, precision=None):
        """Neural flux on (w: float64 CUDA tensor of JS_NN_NPARAM parameters, kept by
        reference: later updates in place take effect; norm: mean[4], sd[4], scale[4] of the
        frame channels; w_bar: float64 CUDA tensor that reverse calls add the parameter
        gradient to, or None; precision: "fp64", "fp32", "bf16" (tensor-core layers; the
        network in one fused launch where no reverse pass reads its activations) or
        "bf16-layerwise" (the same results, one launch per layer); fp32=True is
        precision="fp32") or off (w = None)."""
        if w is None:
            _check(lib().js_set_neural(self.ctx, None, None, None, 0), "js_set_neural")
            self._nn = None
            return
        if w.numel() != JS_NN_NPARAM or (w_bar is not None and w_bar.numel() != JS_NN_NPARAM):
            raise ValueError("w and w_bar hold %d parameters" % JS_NN_NPARAM)
        nm = np.ascontiguousarray(np.asarray(norm, dtype=np.float64).reshape(12))
        prec = precision or ("fp32" if fp32 else "fp64")
        code = {"fp64": JS_NN_F64, "fp32": JS_NN_F32, "bf16": JS_NN_BF16,
                "bf16-layerwise": JS_NN_BF16 | JS_NN_LAYERWISE}[prec]
        _check(lib().js_set_neural(self.ctx, _ptr(w), None if w_bar is None else _ptr(w_bar),
                                   nm.ctypes.data_as(C.c_void_p), code), "js_set_neural")
        self._nn = (w, w_bar, nm)  # keep the device buffers alive while the library uses them

    def set_arith(self, mode):
        """"fast" (default: the fused stage kernel) or "ieee" (every operation IEEE-rounded in
        the canonical order: bit-reproducible)."""
        code = {"fast": JS_ARITH_FAST, "ieee": JS_ARITH_IEEE}[mode]
        _check(lib().js_set_arith(self.ctx, code), "js_set_arith")

    def arith(self):
        m = C.c_int(0)
        _check(lib().js_get_arith(self.ctx, C.byref(m)), "js_get_arith")
        return {JS_ARITH_FAST: "fast", JS_ARITH_IEEE: "ieee"}[m.value]

    def set_tuning(self, variant):
        _check(lib().js_set_tuning(self.ctx, int(variant)), "js_set_tuning")

    def tuning(self):
        v, n = C.c_int(0), C.c_int(0)
        _check(lib().js_get_tuning(self.ctx, C.byref(v), C.byref(n)), "js_get_tuning")
        return v.value, n.value

    def prim_to_cons(self, W):
        import torch
        U = torch.empty_like(W)
        js_prim_to_cons(self.ctx, W, U)
        return U

    def rhs(self, U, out=None):
        import torch
        out = torch.empty_like(U) if out is None else out
        js_rhs(self.ctx, U, out)
        return out

    def max_dt(self, U, cfl):
        return js_max_dt(self.ctx, U, cfl)

    def step(self, U, dt, n_steps=1):
        js_step(self.ctx, U, dt, n_steps)
        return U

    def step_cfl(self, U, cfl, n_steps=1, t=None, t_end=0.0, dt_log=None):
        """n_steps SSP-RK3 steps of the device-computed CFL step size (no host synchronisation);
        t: optional float64 CUDA scalar tensor of the running time (advanced; steps stop at
        t_end > 0); dt_log: optional float64 CUDA tensor of n_steps step sizes."""
        _check(lib().js_step_cfl(self.ctx, _ptr(U), float(cfl), int(n_steps), None if t is None else _ptr(t),
                                 float(t_end), None if dt_log is None else _ptr(dt_log)), "js_step_cfl")

    def rhs_vjp(self, U, lam, U_bar=None, p_bar=None):
        import torch
        U_bar = torch.empty_like(U) if U_bar is None else U_bar
        p_bar = torch.zeros(JS_NPARAM, dtype=torch.float64, device=U.device) if p_bar is None else p_bar
        js_rhs_vjp(self.ctx, U, lam, U_bar, p_bar)
        return U_bar, p_bar

    def step_vjp(self, U_n, dt, lam_np1, lam_n=None, p_bar=None):
        import torch
        lam_n = torch.empty_like(U_n) if lam_n is None else lam_n
        p_bar = torch.zeros(JS_NPARAM, dtype=torch.float64, device=U_n.device) if p_bar is None else p_bar
        js_step_vjp(self.ctx, U_n, dt, lam_np1, lam_n, p_bar)
        return lam_n, p_bar

    def step_stage(self, U_n, U_in, U_out, dt, k, internals=False):
        """One SSP-RK3 stage k (0, 1, 2): U_out = a_k U_n + b_k (U_in + dt L(U_in)); internals:
        also store the stage's WENO5 internals for step_stage_vjp (stages 0, 1)."""
        flag = JS_STAGE_INTERNALS if internals else 0
        _check(lib().js_step_stage(self.ctx, _ptr(U_n) if k > 0 else None, _ptr(U_in), _ptr(U_out), float(dt),
                                   int(k) | flag), "js_step_stage")
        return U_out

    def step_stage_vjp(self, U_in, dt, k, lam_out, lam_in, p_bar=None, internals=False):
        """Reverse of stage k (called for k = 2, 1, 0 of one step; stage 0 adds the U^n part);
        internals: use the internals step_stage stored for this stage."""
        flag = JS_STAGE_INTERNALS if internals else 0
        _check(lib().js_step_stage_vjp(self.ctx, _ptr(U_in), float(dt), int(k) | flag, _ptr(lam_out),
                                       _ptr(lam_in), _ptr(p_bar)), "js_step_stage_vjp")
        return lam_in

    def rows_pack(self, U, row0, nrows, buf, zero=False):
        _check(lib().js_rows_pack(self.ctx, _ptr(U), int(row0), int(nrows), _ptr(buf), int(bool(zero))),
               "js_rows_pack")
        return buf

    def rows_unpack(self, U, row0, nrows, buf, add=False):
        _check(lib().js_rows_unpack(self.ctx, _ptr(U), int(row0), int(nrows), _ptr(buf), int(bool(add))),
               "js_rows_unpack")
        return U

    def tape_reserve(self, n_slots, weno=False):
        """n_slots tape slots; weno=True also records the WENO5 internals of each stage
        (2D grids), so that step_vjp_taped skips their recompute."""
        _check(lib().js_tape_reserve_ex(self.ctx, int(n_slots), JS_TAPE_WENO if weno else 0),
               "js_tape_reserve_ex")

    def nn_eval(self, X):
        """The neural network alone on a normalised image X [4, H, W] (float64 CUDA)."""
        import torch
        X = X.contiguous()
        Y = torch.empty_like(X)
        _check(lib().js_nn_eval(self.ctx, _ptr(X), X.shape[1], X.shape[2], _ptr(Y)), "js_nn_eval")
        return Y

    def nn_eval_vjp(self, X, GY):
        """Reverse of nn_eval: the input gradient for the output gradient GY [4, H, W]; the
        weight gradient is added to the w_bar given to set_neural."""
        import torch
        X, GY = X.contiguous(), GY.contiguous()
        GX = torch.empty_like(X)
        _check(lib().js_nn_eval_vjp(self.ctx, _ptr(X), X.shape[1], X.shape[2], _ptr(GY), _ptr(GX)),
               "js_nn_eval_vjp")
        return GX

    def tape_weno_bytes(self, n_slots):
        """Device bytes the WENO5 internals of n_slots tape slots take (0 on 1D grids)."""
        nx, ny = self._spec["nx"], self._spec["ny"]
        if ny == 1:
            return 0
        pitch = (nx + 6 + 3) // 4 * 4
        plane = max((nx + 6) * ((ny + 6 + 3) // 4 * 4), (pitch * (ny + 6) + 31) // 32 * 32)
        return int(n_slots) * 3 * 56 * 8 * ((plane + 31) // 32 * 32)

    def step_taped(self, U, dt, slot):
        _check(lib().js_step_taped(self.ctx, _ptr(U), float(dt), int(slot)), "js_step_taped")
        return U

    def step_vjp_taped(self, slot, dt, lam_np1, lam_n=None, p_bar=None):
        import torch
        lam_n = torch.empty_like(lam_np1) if lam_n is None else lam_n
        p_bar = torch.zeros(JS_NPARAM, dtype=torch.float64, device=lam_np1.device) if p_bar is None else p_bar
        _check(lib().js_step_vjp_taped(self.ctx, int(slot), float(dt), _ptr(lam_np1), _ptr(lam_n), _ptr(p_bar)),
               "js_step_vjp_taped")
        return lam_n, p_bar

    def status(self):
        return js_sync_status(self.ctx)

    def check(self):
        _check(self.status(), "device status")

    def ib_info(self):
        return js_ib_info(self.ctx, self.nx, self.ny)

    def close(self):
        if getattr(self, "ctx", None):
            js_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------------------
# batched path: one persistent launch advances many independent problems
# ---------------------------------------------------------------------------------------
class Batch:
    """Independent 2D problems advanced together by js_batch_step (one persistent launch)."""

    def __init__(self, problems, stream=None):
        n = len(problems)
        grids = (JsGrid * n)()
        params = (JsParams * n)()
        bcs = (JsBoundary * n)()
        sdfs = (C.c_void_p * n)()
        self._keep = []
        for k, p in enumerate(problems):
            g, pp, b = make_structs(p.nx, p.ny, p.x0, p.y0, p.dx, p.dy, p.bc, p.gamma, p.mu, p.Pr, p.nu, p.inflow,
                                    getattr(p, "wall", 0))
            grids[k], params[k], bcs[k] = g, pp, b
            if p.sdf is not None:
                a = np.ascontiguousarray(p.sdf, dtype=np.float64)
                self._keep.append(a)
                sdfs[k] = a.ctypes.data_as(C.c_void_p)
        out = C.c_void_p()
        _check(lib().js_batch_create(n, grids, params, bcs, sdfs, _stream_ptr(stream), C.byref(out)),
               "js_batch_create")
        self.handle = out
        self.count = n
        self.shapes = [(4, p.ny, p.nx) for p in problems]

    def set_states(self, states):
        if len(states) != self.count:
            raise ValueError("one state per instance")
        ptrs = (C.c_void_p * self.count)(*[_ptr(t).value for t in states])
        self._states = list(states)
        _check(lib().js_batch_set_states(self.handle, ptrs), "js_batch_set_states")

    def step(self, cfl, n_steps, t=None, dt_log=None):
        _check(lib().js_batch_step(self.handle, float(cfl), int(n_steps), _ptr(t), _ptr(dt_log)), "js_batch_step")

    def step_vjp(self, U_n, dts, lam_np1, lam_n, p_bar=None):
        """Reverse of one batched step; lists of per-instance tensors, dts: per-instance floats."""
        n = self.count
        arr = lambda ts: (C.c_void_p * n)(*[_ptr(t).value for t in ts])
        dt = (C.c_double * n)(*[float(x) for x in dts])
        pb = arr(p_bar) if p_bar is not None else None
        _check(lib().js_batch_step_vjp(self.handle, arr(U_n), dt, arr(lam_np1), arr(lam_n), pb), "js_batch_step_vjp")

    def set_tuning(self, blocks_per_sm=0, schedule=0):
        _check(lib().js_batch_set_tuning(self.handle, int(blocks_per_sm), int(schedule)), "js_batch_set_tuning")

    def tuning(self):
        """(blocks per SM, most blocks per SM, schedule, number of schedules)"""
        v = [C.c_int(0) for _ in range(4)]
        _check(lib().js_batch_get_tuning(self.handle, *[C.byref(x) for x in v]), "js_batch_get_tuning")
        return tuple(x.value for x in v)

    def set_reverse_launch(self, split):
        """Launch form of the batched reverse step: 0 one persistent launch, 1 one launch per
        phase (identical results)."""
        _check(lib().js_batch_set_reverse_launch(self.handle, int(split)), "js_batch_set_reverse_launch")

    def reverse_launch(self):
        v = C.c_int(0)
        _check(lib().js_batch_get_reverse_launch(self.handle, C.byref(v)), "js_batch_get_reverse_launch")
        return v.value

    def step_fixed(self, dts):
        """Advance every registered state len(dts) steps of the given sizes: dts float64 CUDA
        tensor [n_steps, count]."""
        _check(lib().js_batch_step_fixed(self.handle, int(dts.shape[0]), _ptr(dts)), "js_batch_step_fixed")

    def rollout_spacing(self, n_steps):
        """The checkpoint spacing rollout_forward / rollout_vjp use for n_steps with ckpt=0."""
        c = C.c_int(0)
        _check(lib().js_batch_rollout_spacing(self.handle, int(n_steps), C.byref(c)), "js_batch_rollout_spacing")
        return c.value

    def rollout_forward(self, cfl, dt_log, ckpt=0):
        """Advance the registered states dt_log.shape[0] CFL steps, logging the step sizes into
        dt_log (float64 CUDA tensor [n_steps, count]) and keeping checkpoints for rollout_vjp."""
        _check(lib().js_batch_rollout_forward(self.handle, float(cfl), int(dt_log.shape[0]), int(ckpt), _ptr(dt_log)),
               "js_batch_rollout_forward")

    def rollout_vjp(self, dt_log, lam, p_bar=None, ckpt=0):
        """Reverse of the rollout from the registered states with the step sizes dt_log
        (float64 CUDA tensor [n_steps, count]); lam: per-instance tensors, dL/dU_N in, dL/dU_0
        out; p_bar: per-instance JS_NPARAM tensors (accumulated) or None; ckpt: checkpoint
        spacing (0: rollout_spacing's choice)."""
        n = self.count
        arr = lambda ts: (C.c_void_p * n)(*[_ptr(t).value for t in ts])
        pb = arr(p_bar) if p_bar is not None else None
        _check(lib().js_batch_rollout_vjp(self.handle, int(dt_log.shape[0]), _ptr(dt_log), int(ckpt), arr(lam), pb),
               "js_batch_rollout_vjp")

    def status(self):
        return lib().js_batch_sync_status(self.handle)

    def info(self):
        b, t, c = C.c_int(0), C.c_int(0), C.c_longlong(0)
        _check(lib().js_batch_info(self.handle, C.byref(b), C.byref(t), C.byref(c)), "js_batch_info")
        return dict(blocks=b.value, tiles=t.value, cells=c.value)

    def test_timeout(self, budget_s):
        _check(lib().js_batch_test_timeout(self.handle, float(budget_s)), "js_batch_test_timeout")

    def close(self):
        if getattr(self, "handle", None):
            lib().js_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def block_average(U, fx, fy=1, stream=None):
    """Means of fx x fy cell blocks of a float64 CUDA state [4, ny, nx] (js_block_average)."""
    import torch
    U = U.contiguous()
    ny, nx = U.shape[1], U.shape[2]
    out = torch.empty((4, ny // fy, nx // fx), dtype=torch.float64, device=U.device)
    _check(lib().js_block_average(_ptr(U), nx, ny, int(fx), int(fy), _ptr(out), _stream_ptr(stream)),
           "js_block_average")
    return out

