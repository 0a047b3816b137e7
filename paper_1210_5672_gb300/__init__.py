"""GB300 (sm_103a) library for the Jacobian of the standing-water-wave shooting
map (Wilkening & Yu, overdetermined shooting methods, Sec. 3.3).

This module is a thin ctypes binding of the C ABI in ``include/ww.h``: it
marshals torch CUDA tensors (device pointers) and numpy arrays (host pointers)
into the library calls and turns negative status codes into exceptions.  No
step of the method runs in Python; if the compiled library is missing the
import of any entry point raises.

Names follow the C ABI: ``dtn_setup``, ``dtn_apply``, ``shoot``,
``shoot_jacobian``, ``shoot_jacobian_host``, ``shoot_jacobian_batch``,
``objective_and_grad``, plus the
``Context`` that owns the device workspace and ``ShootingObjective``, a
``torch.autograd.Function`` around ``objective_and_grad``.

Layouts: every array is float64; matrices are column-major with leading
dimension N, so an N x m matrix is passed as a contiguous torch tensor of
shape (m, N) (row j = column j of the matrix).
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libww.so")

WW_OK = 0
ERRORS = {
    -1: "WW_ERR_ARG", -2: "WW_ERR_GEOMETRY", -3: "WW_ERR_NO_CONVERGENCE",
    -4: "WW_ERR_CUDA", -5: "WW_ERR_TIMEOUT", -6: "WW_ERR_ALLOC",
}
WW_FP64, WW_MIXED = 0, 1
EXPORTS = ("ww_create", "ww_destroy", "ww_set_stream", "ww_get_stats", "ww_last_error", "ww_set_timing",
           "ww_get_timing", "dtn_setup", "dtn_apply", "shoot", "shoot_jacobian", "shoot_jacobian_host",
           "shoot_jacobian_batch", "objective_and_grad", "dtn_apply_static", "ww_set_verify", "ww_set_checkpoint", "ww_set_schedule", "ww_get_schedule",
           "ww_autotune", "ww_set_segment", "shoot_jacobian_segments", "objective_and_grad_segments",
           "ww_selftest_f32gemm",
           "ww_selftest_ozaki", "ww_selftest_dgemm", "ww_selftest_recip")
STATIC_MAX_N, STATIC_MAX_RHS = 256, 64
PHASES = ("assembly", "factor", "solve", "gapply", "colrhs", "gamma", "base", "gkernel", "inverse")


class WWError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _Problem(C.Structure):
    _fields_ = [
        ("N", C.c_int), ("n", C.c_int), ("g", C.c_double), ("tau", C.c_double), ("h", C.c_double),
        ("steps", C.c_int), ("basis", C.POINTER(C.c_double)), ("precision", C.c_int),
        ("refine_tol", C.c_double), ("max_refine", C.c_int),
    ]


class Schedule(C.Structure):
    """ww_schedule: the knobs of the step program (see include/ww.h)."""
    _fields_ = [("overlap", C.c_int), ("ns_every", C.c_int), ("corr_bn", C.c_int), ("inv_bn", C.c_int),
                ("lu_nb", C.c_int), ("inv_ctas", C.c_int), ("prio", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class _Segment(C.Structure):
    _fields_ = [("steps", C.c_int), ("theta", C.c_double), ("rho", C.c_double), ("centre", C.c_int),
                ("stages", C.c_int), ("a", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double))]


class Stats(C.Structure):
    _fields_ = [
        ("refine_iters_max", C.c_int), ("refine_resid_max", C.c_double), ("ns_resid_max", C.c_double),
        ("stages", C.c_int), ("launches", C.c_longlong), ("refine_iters_mean", C.c_double),
        ("refine_resid_measured", C.c_double), ("verified_solves", C.c_int),
        ("device_bytes", C.c_longlong), ("adjoint_bytes", C.c_longlong),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load the compiled library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; "
                               "g.build()')")
        L = C.CDLL(LIB_PATH)
        V, I, D = C.c_void_p, C.c_int, C.c_double
        sig = {
            "ww_create": (I, [C.POINTER(V), C.POINTER(_Problem)]),
            "ww_destroy": (None, [V]),
            "ww_set_stream": (I, [V, V]),
            "ww_get_stats": (I, [V, C.POINTER(Stats)]),
            "ww_last_error": (C.c_char_p, []),
            "ww_set_timing": (I, [V, I]),
            "ww_get_timing": (I, [V, C.POINTER(C.c_double), C.POINTER(C.c_int)]),
            "dtn_setup": (I, [V, V]),
            "dtn_apply": (I, [V, V, I, V]),
            "shoot": (I, [V, V, V, V]),
            "shoot_jacobian": (I, [V, V, V, V, V]),
            "shoot_jacobian_host": (I, [V, V, V, V, V]),
            "shoot_jacobian_batch": (I, [C.POINTER(V), I, C.POINTER(V), C.POINTER(V), C.POINTER(V),
                                         C.POINTER(V)]),
            "objective_and_grad": (I, [V, V, V, V]),
            "dtn_apply_static": (I, [V, V, I, I, D, V, V]),
            "ww_set_verify": (I, [V, I]),
            "ww_set_checkpoint": (I, [V, I]),
            "ww_set_schedule": (I, [V, C.POINTER(Schedule)]),
            "ww_get_schedule": (I, [V, C.POINTER(Schedule)]),
            "ww_autotune": (I, [V, V, I, C.c_char_p, C.POINTER(D)]),
            "ww_set_segment": (I, [V, C.POINTER(_Segment)]),
            "shoot_jacobian_segments": (I, [C.POINTER(V), I, V, V, V, V]),
            "objective_and_grad_segments": (I, [C.POINTER(V), I, V, V, V]),
            "ww_selftest_f32gemm": (I, [V, V, I, I, I, V]),
            "ww_selftest_ozaki": (I, [V, V, I, I, I, V]),
            "ww_selftest_dgemm": (I, [V, V, I, I, I, V]),
            "ww_selftest_recip": (I, [V, I, C.POINTER(D)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code: int):
    if code != WW_OK:
        raise WWError(code, lib().ww_last_error().decode())


def _dptr(t, numel: int, name: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name}: expected a contiguous float64 CUDA tensor")
    if t.numel() < numel:
        raise ValueError(f"{name}: needs at least {numel} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def _hptr(a: np.ndarray, numel: int, name: str):
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError(f"{name}: expected a contiguous float64 numpy array")
    if a.size < numel:
        raise ValueError(f"{name}: needs at least {numel} elements, got {a.size}")
    return C.c_void_p(a.ctypes.data)


class Context:
    """Owns a ww_ctx (device workspace for one problem size) on the current device."""

    def __init__(self, N, n, g=1.0, tau=0.0, h=1.0, steps=64, basis=None, precision=WW_FP64,
                 refine_tol=0.0, max_refine=0):
        self.N, self.n, self.steps = int(N), int(n), int(steps)
        self.g, self.tau, self.h = float(g), float(tau), float(h)
        self.precision = int(precision)
        self._basis = None
        bp = C.cast(None, C.POINTER(C.c_double))
        if basis is not None:
            b = np.asarray(basis, dtype=np.float64)
            if b.shape != (2 * self.N, self.n):
                raise ValueError("basis must have shape (2N, n)")
            self._basis = np.ascontiguousarray(b.T)   # column-major 2N x n
            bp = self._basis.ctypes.data_as(C.POINTER(C.c_double))
        p = _Problem(self.N, self.n, self.g, self.tau, self.h, self.steps, bp, self.precision,
                     float(refine_tol), int(max_refine))
        h_ = C.c_void_p()
        _check(lib().ww_create(C.byref(h_), C.byref(p)))
        self._h = h_

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("context is closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().ww_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream):
        """Queue work on a torch.cuda.Stream (or raw cudaStream_t int)."""
        raw = getattr(stream, "cuda_stream", stream)
        _check(lib().ww_set_stream(self.handle, C.c_void_p(int(raw) if raw else None)))

    def set_timing(self, enable: bool):
        _check(lib().ww_set_timing(self.handle, 1 if enable else 0))

    def set_checkpoint(self, every: int):
        """objective_and_grad memory: 0 keeps every stage's record; K > 0 keeps
        the base state every K steps and recomputes each segment's records
        (K = round(sqrt(steps)) bounds the memory by ~sqrt(steps))."""
        _check(lib().ww_set_checkpoint(self.handle, int(every)))

    def schedule(self) -> dict:
        sch = Schedule()
        _check(lib().ww_get_schedule(self.handle, C.byref(sch)))
        return sch.as_dict()

    def set_schedule(self, **kw):
        """Change fields of the schedule (overlap, ns_every, corr_bn, inv_bn, lu_nb, inv_ctas, prio)."""
        cur = self.schedule()
        unknown = set(kw) - set(cur)
        if unknown:
            raise ValueError(f"unknown schedule fields {sorted(unknown)}")
        cur.update(kw)
        _check(lib().ww_set_schedule(self.handle, C.byref(Schedule(**cur))))

    def autotune(self, c, probe_steps: int = 4, cache_path=None) -> float:
        """ww_autotune on the shot c (CUDA float64, n+1): the fastest schedule is
        kept (and appended to cache_path); returns its probe ms per RK step
        (0.0 when the choice came from the cache)."""
        ms = C.c_double(0.0)
        path = None if cache_path is None else os.fsencode(cache_path)
        _check(lib().ww_autotune(self.handle, _dptr(c, self.n + 1, "c"), int(probe_steps), path, C.byref(ms)))
        return ms.value

    def set_verify(self, every: int):
        """WW_MIXED: measure the true refinement residual of every `every`-th
        multi-column solve (stats()['refine_resid_measured']); 0 turns it off."""
        _check(lib().ww_set_verify(self.handle, int(every)))

    def timing(self) -> dict:
        """{phase: (total_ms, launches)} of the last shoot / shoot_jacobian."""
        ms = (C.c_double * len(PHASES))()
        cnt = (C.c_int * len(PHASES))()
        _check(lib().ww_get_timing(self.handle, ms, cnt))
        return {p: (ms[i], cnt[i]) for i, p in enumerate(PHASES)}

    def stats(self) -> dict:
        s = Stats()
        _check(lib().ww_get_stats(self.handle, C.byref(s)))
        return s.as_dict()

    # convenience allocation of outputs on the current CUDA device
    def empty_outputs(self):
        import torch
        r = torch.empty(self.N, dtype=torch.float64, device="cuda")
        J = torch.empty(self.n + 1, self.N, dtype=torch.float64, device="cuda")
        f = torch.empty(1, dtype=torch.float64, device="cuda")
        return r, J, f


# ------------------------------------------------------------- entry points
def dtn_setup(ctx: Context, eta):
    """Assemble and factor the DtN operator of the surface eta (CUDA, N)."""
    _check(lib().dtn_setup(ctx.handle, _dptr(eta, ctx.N, "eta")))


def dtn_apply(ctx: Context, phi, Gphi=None):
    """G phi for nrhs columns: phi is (nrhs, N) or (N,) CUDA float64."""
    import torch
    nrhs = 1 if phi.dim() == 1 else phi.shape[0]
    if Gphi is None:
        Gphi = torch.empty_like(phi)
    _check(lib().dtn_apply(ctx.handle, _dptr(phi, nrhs * ctx.N, "phi"), int(nrhs),
                           _dptr(Gphi, nrhs * ctx.N, "Gphi")))
    return Gphi


def shoot(ctx: Context, c, r, f):
    _check(lib().shoot(ctx.handle, _dptr(c, ctx.n + 1, "c"), _dptr(r, ctx.N, "r"), _dptr(f, 1, "f")))


def shoot_jacobian(ctx: Context, c, r, J, f):
    """J: (n+1, N) CUDA float64 (= N x (n+1) column-major)."""
    _check(lib().shoot_jacobian(ctx.handle, _dptr(c, ctx.n + 1, "c"), _dptr(r, ctx.N, "r"),
                                _dptr(J, ctx.N * (ctx.n + 1), "J"), _dptr(f, 1, "f")))


def shoot_jacobian_host(ctx: Context, c: np.ndarray, r: np.ndarray, J: np.ndarray, f: np.ndarray):
    """Host-array variant; J is (n+1, N) float64 (= N x (n+1) column-major)."""
    _check(lib().shoot_jacobian_host(ctx.handle, _hptr(c, ctx.n + 1, "c"), _hptr(r, ctx.N, "r"),
                                     _hptr(J, ctx.N * (ctx.n + 1), "J"), _hptr(f, 1, "f")))


def shoot_jacobian_batch(ctxs, cs, rs, Js, fs):
    """Independent shots run concurrently (one stream each): lists of contexts
    and of each shot's c, r, J (n+1, N) and f CUDA float64 tensors."""
    n = len(ctxs)
    if not (len(cs) == len(rs) == len(Js) == len(fs) == n):
        raise ValueError("shoot_jacobian_batch: one c, r, J, f per context")
    arr = C.c_void_p * max(n, 1)
    hs = arr(*[x.handle for x in ctxs])
    cp = arr(*[_dptr(c, x.n + 1, "c") for x, c in zip(ctxs, cs)])
    rp = arr(*[_dptr(r, x.N, "r") for x, r in zip(ctxs, rs)])
    Jp = arr(*[_dptr(J, x.N * (x.n + 1), "J") for x, J in zip(ctxs, Js)])
    fp = arr(*[_dptr(f, 1, "f") for x, f in zip(ctxs, fs)])
    _check(lib().shoot_jacobian_batch(hs, n, cp, rp, Jp, fp))


def objective_and_grad(ctx: Context, c, f, grad):
    """f (1,) and grad (n+1,) CUDA float64 by the discrete adjoint (grad[0] = d f / d T)."""
    _check(lib().objective_and_grad(ctx.handle, _dptr(c, ctx.n + 1, "c"), _dptr(f, 1, "f"),
                                    _dptr(grad, ctx.n + 1, "grad")))


def dtn_apply_static(eta, phi, h, Gphi, stream=None):
    """G phi without any allocation (fixed workspace inside the library):
    eta (N,), phi and Gphi (nrhs, N) CUDA float64; N <= STATIC_MAX_N,
    nrhs <= STATIC_MAX_RHS."""
    N = eta.numel()
    nrhs = 1 if phi.dim() == 1 else phi.shape[0]
    raw = getattr(stream, "cuda_stream", stream)
    _check(lib().dtn_apply_static(_dptr(eta, N, "eta"), _dptr(phi, N * nrhs, "phi"), int(N), int(nrhs),
                                  float(h), _dptr(Gphi, N * nrhs, "Gphi"), C.c_void_p(int(raw) if raw else None)))
    return Gphi


def tableau(name: str):
    """(a, b) of an explicit Runge-Kutta scheme: 'rk4' (classic) or 'dop853'
    (Dormand and Prince's 8th-order scheme, the paper's integrator: its 12
    stages and 8th-order weights, read from scipy's table of the published
    coefficients)."""
    if name == "rk4":
        a = np.zeros((4, 4))
        a[1, 0], a[2, 1], a[3, 2] = 0.5, 0.5, 1.0
        return a, np.array([1.0, 2.0, 2.0, 1.0]) / 6.0
    if name == "dop853":
        from scipy.integrate._ivp import dop853_coefficients as d
        s = d.N_STAGES
        return np.array(d.A[:s, :s], dtype=np.float64), np.array(d.B, dtype=np.float64)
    raise ValueError(f"unknown tableau {name!r}")


def set_segment(ctx: Context, steps: int, theta: float, rho: float = 1.0, centre: int = 1, scheme="dop853"):
    """Make ctx (N = the segment's M) a segment of a segmented shot (Sec. 2.2):
    `steps` uniform steps of `scheme` ('rk4', 'dop853' or an (a, b) pair) over
    the fraction theta of T/4 on the mesh of Eq. (xi) with parameter rho,
    refined near x = pi (centre 1) or x = 0 (centre 0)."""
    a, b = tableau(scheme) if isinstance(scheme, str) else scheme
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
    if a.shape != (b.size, b.size):
        raise ValueError("tableau: a must be s x s and b of length s")
    sg = _Segment(int(steps), float(theta), float(rho), int(centre), int(b.size),
                  a.ctypes.data_as(C.POINTER(C.c_double)), b.ctypes.data_as(C.POINTER(C.c_double)))
    _check(lib().ww_set_segment(ctx.handle, C.byref(sg)))


def shoot_jacobian_segments(ctxs, c, r, J, f):
    """The segmented shot through the contexts of its segments (in time order):
    r (M_last,), J (n+1, M_last) and f (1,) CUDA float64; c (n+1,) on ctxs[0]'s device."""
    last = ctxs[-1]
    arr = (C.c_void_p * len(ctxs))(*[x.handle for x in ctxs])
    _check(lib().shoot_jacobian_segments(arr, len(ctxs), _dptr(c, ctxs[0].n + 1, "c"), _dptr(r, last.N, "r"),
                                         _dptr(J, last.N * (last.n + 1), "J"), _dptr(f, 1, "f")))


def objective_and_grad_segments(ctxs, c, f, grad):
    """f (1,) and grad (n+1,) CUDA float64 of the segmented shot by its discrete
    adjoint (grad[0] = d f / d T); contexts as shoot_jacobian_segments."""
    arr = (C.c_void_p * len(ctxs))(*[x.handle for x in ctxs])
    n = ctxs[0].n
    _check(lib().objective_and_grad_segments(arr, len(ctxs), _dptr(c, n + 1, "c"), _dptr(f, 1, "f"),
                                             _dptr(grad, n + 1, "grad")))


def selftest(kind: str, A, B):
    """The library's product A @ B (A: M x K, B: K x Nn CUDA float64 tensors) as
    an (M, Nn) CUDA tensor; kind 'f32gemm' (3 + 3 bf16 slices, tensor cores),
    'ozaki' (7 + 7 exact bf16 digits, tensor cores) or 'dgemm' (FP64 DGEMM)."""
    import torch
    M, K = A.shape
    K2, Nn = B.shape
    assert K == K2
    At = A.t().contiguous()   # column-major storage
    Bt = B.t().contiguous()
    Ct = torch.empty(Nn, M, dtype=torch.float64, device=A.device)
    fn = {"f32gemm": lib().ww_selftest_f32gemm, "ozaki": lib().ww_selftest_ozaki,
          "dgemm": lib().ww_selftest_dgemm}[kind]
    _check(fn(_dptr(At, M * K, "A"), _dptr(Bt, K * Nn, "B"), M, Nn, K, _dptr(Ct, M * Nn, "C")))
    return Ct.t()


def selftest_recip(d) -> float:
    """max relative difference of the assembly's reciprocal from 1/d over the
    positive CUDA float64 tensor d."""
    out = C.c_double(-1.0)
    _check(lib().ww_selftest_recip(_dptr(d, d.numel(), "d"), int(d.numel()), C.byref(out)))
    return out.value


def _autograd_fn():
    import torch

    class ShootingObjective(torch.autograd.Function):
        """f(c) = |r(c)|^2 / 2 with d f / d c from objective_and_grad."""

        @staticmethod
        def forward(ctx_, c, wwctx):
            cc = c.detach().contiguous()
            f = torch.empty(1, dtype=torch.float64, device=c.device)
            grad = torch.empty(wwctx.n + 1, dtype=torch.float64, device=c.device)
            objective_and_grad(wwctx, cc, f, grad)
            ctx_.save_for_backward(grad)
            return f[0]

        @staticmethod
        def backward(ctx_, gout):
            (grad,) = ctx_.saved_tensors
            return gout * grad, None

    return ShootingObjective


def shooting_objective(c, wwctx: Context):
    """Differentiable objective f(c) (torch autograd), gradient from the library."""
    return _autograd_fn().apply(c, wwctx)


def default_basis(N: int, n: int) -> np.ndarray:
    """(2N, n) basis of the default initial data: column k = (cos(k x), 0)."""
    x = 2.0 * math.pi * np.arange(N) / N
    B = np.zeros((2 * N, n))
    for k in range(1, n + 1):
        B[:N, k - 1] = np.cos(k * x)
    return B
