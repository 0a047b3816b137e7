"""CPU FP64 oracle for the standing-wave shooting Jacobian (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never touches it, and the two share no code.

The arithmetic lives in ``ww_oracle.c`` (plain C99, IEEE double, optional
OpenMP over independent rows/columns).  This module compiles it with gcc on
first use and exposes thin numpy wrappers.  Each wrapper names the passage of
the paper the C function follows:

* ``fft``            -- textbook radix-2 DFT used for every spectral step
* ``spectral``       -- Fourier multipliers: d/dx, Hilbert (-i sgn k),
                        36th-order filter (Eq. filter), projection P
* ``dtn_matrices``   -- A = 1/2 I + K and G of Eq. (K1K2) (image sign: reading R1)
* ``dtn``            -- Dirichlet-to-Neumann operator, Eqs. (fred), (G)
* ``rhs``            -- Eq. (ww) base RHS and Eqs. (l5a), (l6a) variational RHS
* ``shoot``          -- r and f of Eq. (f:phi)
* ``shoot_jacobian`` -- J of Eqs. (Jik), (q:qdot), T column by reading R2
* ``objective_and_grad`` -- f and its gradient by the discrete adjoint of the
                        RK4 scheme (Sec. 3.2 Eqs. adj, nabla:f; App. C Eq. adj2;
                        reading R18: exact transpose of the discrete map)
* ``dtn_T``          -- the transpose of the discrete DtN operator
* ``energy``         -- the energy monitor of Sec. 4
* ``mesh``, ``mesh_inverse``, ``interp`` -- the change of variables of Eq. (xi)
                        (Eq. rho:def), its inverse by Newton's method and the
                        trigonometric interpolant used to respace (Sec. 2.2)
* ``tableau``        -- explicit Runge-Kutta tableaux: classic RK4, and DOP853
                        (Dormand and Prince's 8th-order 12-stage scheme of Sec.
                        2.2, the published coefficients as scipy ships them)
* ``shoot_segments``, ``shoot_jacobian_segments``, ``evolve_segments`` -- the
                        shot over time segments with their own grids, meshes
                        and step counts (Sec. 2.2), any tableau
* ``rhs_segment``, ``dtn_segment`` -- the RHS and the DtN on a segment's mesh
* ``objective_and_grad_segments``, ``rhs_T_segment`` -- the discrete adjoint of
                        the segmented shot (reading R18 carried to meshes,
                        respacing and any tableau) and its transposed RHS
* ``wide_*``         -- the same C compiled with long double (x87 extended on
                        x86-64, binary128 on aarch64): the double build's own
                        rounding error on the same discrete map
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ww_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libww_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, plant: int = 0, wide: bool = False) -> str:
    """Compile ww_oracle.c into oracle/_build/libww_oracle.so (gcc -O2 -fopenmp).
    plant > 0 builds a deliberately wrong variant (tests of the pins only);
    wide builds the same arithmetic in long double (ORC_WIDE)."""
    os.makedirs(_BUILD, exist_ok=True)
    lib_path = _LIB if plant == 0 else os.path.join(_BUILD, f"libww_oracle_plant{plant}.so")
    if wide:
        lib_path = os.path.join(_BUILD, "libww_oracle_wide.so")
    if force or not os.path.exists(lib_path) or os.path.getmtime(lib_path) < os.path.getmtime(_SRC):
        tmp = lib_path + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", f"-DORC_PLANT={int(plant)}"] + \
              (["-DORC_WIDE"] if wide else []) + [_SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib_path)
    return lib_path


class Problem(C.Structure):
    _fields_ = [
        ("N", C.c_int), ("n", C.c_int), ("g", C.c_double), ("tau", C.c_double),
        ("h", C.c_double), ("steps", C.c_int), ("basis", C.POINTER(C.c_double)),
    ]


_D = C.POINTER(C.c_double)


class Segment(C.Structure):
    """One time segment (Sec. 2.2): M grid points, `steps` uniform steps over
    the fraction theta of T/4, mesh parameter rho of Eq. (xi) (1 = uniform),
    refined near x = pi (centre = 1) or x = 0 (centre = 0)."""
    _fields_ = [("M", C.c_int), ("steps", C.c_int), ("theta", C.c_double), ("rho", C.c_double),
                ("centre", C.c_int)]


class Tableau(C.Structure):
    _fields_ = [("s", C.c_int), ("a", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double))]


def load(path: str):
    """ctypes handle of a compiled oracle with the signatures set."""
    L = C.CDLL(path)
    _set_signatures(L)
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


def _set_signatures(L):
    P = C.POINTER(Problem)
    sig = {
        "orc_fft": (None, [C.c_int, _D, C.c_int]),
        "orc_spectral": (None, [C.c_int, C.c_int, _D, _D]),
        "orc_assemble": (None, [C.c_int, C.c_double, _D, _D, _D, _D, _D]),
        "orc_dtn_matrices": (None, [C.c_int, C.c_double, _D, _D, _D]),
        "orc_dtn": (None, [C.c_int, C.c_double, _D, _D, C.c_int, _D]),
        "orc_lu": (C.c_int, [C.c_int, _D, C.POINTER(C.c_int)]),
        "orc_lu_solve": (None, [C.c_int, _D, C.POINTER(C.c_int), _D, _D]),
        "orc_rhs": (None, [P, C.c_double, _D, C.c_int, C.c_int, _D]),
        "orc_initial": (None, [P, _D, _D]),
        "orc_evolve": (None, [P, C.c_double, _D, _D]),
        "orc_evolve_columns": (None, [P, C.c_double, _D, _D, C.c_int, C.c_int, _D]),
        "orc_shoot": (None, [P, _D, _D, _D]),
        "orc_shoot_jacobian": (None, [P, _D, _D, _D, _D]),
        "orc_energy": (C.c_double, [P, _D]),
        "orc_objective_and_grad": (None, [P, _D, _D, _D]),
        "orc_dtn_T": (None, [C.c_int, C.c_double, _D, _D, _D]),
        "orc_trajectory_columns": (None, [P, C.c_double, _D, _D, C.c_int, C.c_int, _D]),
        "orc_adjoint_trajectory": (None, [P, _D, _D]),
        "orc_lu_solve_T": (None, [C.c_int, _D, C.POINTER(C.c_int), _D, _D]),
        "orc_mesh_eval": (None, [C.c_double, C.c_int, C.c_int, _D, _D, _D]),
        "orc_mesh_inverse": (None, [C.c_double, C.c_int, C.c_int, _D, _D]),
        "orc_interp": (None, [C.c_int, _D, C.c_int, _D, _D]),
        "orc_evolve_segments": (C.c_int, [P, C.c_int, C.POINTER(Segment), C.POINTER(Tableau), C.c_double, _D,
                                          _D]),
        "orc_shoot_segments": (C.c_int, [P, C.c_int, C.POINTER(Segment), C.POINTER(Tableau), _D, _D, _D]),
        "orc_shoot_jacobian_segments": (C.c_int, [P, C.c_int, C.POINTER(Segment), C.POINTER(Tableau), _D, _D,
                                                  _D, _D]),
        "orc_rhs_segment": (None, [P, C.POINTER(Segment), C.c_double, _D, C.c_int, C.c_int, _D]),
        "orc_dtn_segment": (None, [C.POINTER(Segment), C.c_double, _D, _D, _D]),
        "orc_objective_and_grad_segments": (C.c_int, [P, C.c_int, C.POINTER(Segment), C.POINTER(Tableau), _D, _D,
                                                      _D]),
        "orc_rhs_T_segment": (None, [P, C.POINTER(Segment), _D, _D, _D, _D]),
        "orc_energy_segment": (C.c_double, [P, C.POINTER(Segment), _D]),
        "orc_threads": (C.c_int, []),
        "orc_set_threads": (None, [C.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


MUL_DERIV, MUL_HILBERT, MUL_FILTER, MUL_PROJECT = 0, 1, 2, 3


def threads() -> int:
    return lib().orc_threads()


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


def make_problem(N, n, g=1.0, tau=0.0, h=1.0, steps=64, basis=None):
    """Return (Problem, keepalive) -- the basis array must outlive the struct."""
    keep = None
    bp = C.cast(None, _D)
    if basis is not None:
        keep = np.asfortranarray(np.asarray(basis, dtype=np.float64))
        assert keep.shape == (2 * N, n)
        keep = np.ascontiguousarray(keep.T)  # column k contiguous (2N each)
        bp = _p(keep)
    return Problem(int(N), int(n), float(g), float(tau), float(h), int(steps), bp), keep


def fft(x, inverse=False) -> np.ndarray:
    z = np.ascontiguousarray(np.asarray(x, dtype=np.complex128)).copy()
    lib().orc_fft(len(z), z.ctypes.data_as(_D), 1 if inverse else 0)
    return z


def spectral(kind: int, f) -> np.ndarray:
    f = _f64(f)
    out = np.empty_like(f)
    lib().orc_spectral(len(f), int(kind), _p(f), _p(out))
    return out


def dtn_matrices(eta, h):
    """(A, G) row-major N x N: A = 1/2 I + K, Eq. (K1K2) / N."""
    eta = _f64(eta)
    N = len(eta)
    A = np.empty((N, N)); G = np.empty((N, N))
    lib().orc_dtn_matrices(N, float(h), _p(eta), _p(A), _p(G))
    return A, G


def dtn(eta, phi, h) -> np.ndarray:
    """DtN of phi (shape (N,) or (nrhs, N)) on the surface eta, Eqs. (fred), (G)."""
    eta = _f64(eta)
    phi = _f64(phi)
    one = phi.ndim == 1
    phi2 = phi.reshape(1, -1) if one else phi
    out = np.empty_like(phi2)
    lib().orc_dtn(len(eta), float(h), _p(eta), _p(phi2), phi2.shape[0], _p(out))
    return out[0] if one else out


def rhs(prob: Problem, T: float, y, ncol: int, t_col: int = 0) -> np.ndarray:
    """Filtered RHS; y has shape (ncol+1, 2N): row 0 = (eta, phi), rows 1.. = columns."""
    y = _f64(y).reshape(ncol + 1, 2 * prob.N)
    out = np.empty_like(y)
    lib().orc_rhs(C.byref(prob), float(T), _p(y), int(ncol), int(t_col), _p(out))
    return out


def initial(prob: Problem, c) -> np.ndarray:
    c = _f64(c)
    q = np.empty(2 * prob.N)
    lib().orc_initial(C.byref(prob), _p(c), _p(q))
    return q


def evolve(prob: Problem, T: float, q0) -> np.ndarray:
    q0 = _f64(q0)
    out = np.empty_like(q0)
    lib().orc_evolve(C.byref(prob), float(T), _p(q0), _p(out))
    return out


def evolve_columns(prob: Problem, T: float, q0, cols, t_col: int = 0) -> np.ndarray:
    q0 = _f64(q0)
    cols = _f64(cols)
    ncol = cols.shape[0]
    out = np.empty((ncol + 1, 2 * prob.N))
    lib().orc_evolve_columns(C.byref(prob), float(T), _p(q0), _p(cols), ncol, int(t_col), _p(out))
    return out


def shoot(prob: Problem, c):
    c = _f64(c)
    r = np.empty(prob.N); f = np.empty(1)
    lib().orc_shoot(C.byref(prob), _p(c), _p(r), _p(f))
    return r, float(f[0])


def shoot_jacobian(prob: Problem, c):
    """(r, J, f) with J of shape (N, n+1) (column 0 = d r / d T)."""
    c = _f64(c)
    N, n = prob.N, prob.n
    r = np.empty(N); f = np.empty(1)
    Jc = np.empty((n + 1, N))  # column-major storage = row-major of J^T
    lib().orc_shoot_jacobian(C.byref(prob), _p(c), _p(r), _p(Jc), _p(f))
    return r, np.ascontiguousarray(Jc.T), float(f[0])


def objective_and_grad(prob: Problem, c):
    """(f, grad) with grad[0] = d f / d T and grad[k] = d f / d c_k, by the
    discrete adjoint (reading R18)."""
    c = _f64(c)
    f = np.empty(1)
    g = np.empty(prob.n + 1)
    lib().orc_objective_and_grad(C.byref(prob), _p(c), _p(f), _p(g))
    return float(f[0]), g


def trajectory_columns(prob: Problem, T: float, q0, cols, t_col: int = 0) -> np.ndarray:
    """Base state and variational columns at every step boundary: shape
    (steps + 1, ncol + 1, 2N)."""
    q0 = _f64(q0)
    cols = _f64(np.atleast_2d(cols))
    ncol = cols.shape[0]
    out = np.empty((prob.steps + 1, ncol + 1, 2 * prob.N))
    lib().orc_trajectory_columns(C.byref(prob), float(T), _p(q0), _p(cols), ncol, int(t_col), _p(out))
    return out


def adjoint_trajectory(prob: Problem, c) -> np.ndarray:
    """The discrete adjoint state at every step boundary, shape (steps + 1, 2N):
    row n is the gradient of f with respect to the state at the start of step n."""
    c = _f64(c)
    out = np.empty((prob.steps + 1, 2 * prob.N))
    lib().orc_adjoint_trajectory(C.byref(prob), _p(c), _p(out))
    return out


def dtn_T(eta, x, h) -> np.ndarray:
    """The transpose of the discrete DtN operator applied to x."""
    eta = _f64(eta)
    x = _f64(x)
    out = np.empty_like(x)
    lib().orc_dtn_T(len(eta), float(h), _p(eta), _p(x), _p(out))
    return out


def energy(prob: Problem, q) -> float:
    q = _f64(q)
    return float(lib().orc_energy(C.byref(prob), _p(q)))


# ------------------------------------------------------------ segments (Sec. 2.2)
def mesh(rho: float, M: int, centre: int = 1):
    """(x, E, E') of Eq. (xi) at alpha_j = 2 pi j / M: x = xi(alpha_j), E = xi', E' = xi''."""
    x, e, e1 = np.empty(M), np.empty(M), np.empty(M)
    lib().orc_mesh_eval(float(rho), int(centre), int(M), _p(x), _p(e), _p(e1))
    return x, e, e1


def mesh_inverse(rho: float, x, centre: int = 1) -> np.ndarray:
    x = _f64(x)
    out = np.empty_like(x)
    lib().orc_mesh_inverse(float(rho), int(centre), x.size, _p(x), _p(out))
    return out


def interp(f, beta) -> np.ndarray:
    """The trigonometric interpolant of f (values at 2 pi j / M) at the points beta."""
    f, beta = _f64(f), _f64(beta)
    out = np.empty(beta.size)
    lib().orc_interp(f.size, _p(f), beta.size, _p(beta), _p(out))
    return out


def tableau(name: str):
    """(a, b) of an explicit Runge-Kutta scheme: 'rk4' (classic) or 'dop853'.
    DOP853's coefficients are Dormand and Prince's published ones (Hairer,
    Norsett and Wanner, Solving ODEs I), read from scipy's copy of the table:
    its 12 stages and the 8th-order weights; the 13th evaluation of the
    original code serves only its error estimate and dense output."""
    if name == "rk4":
        a = np.zeros((4, 4))
        a[1, 0], a[2, 1], a[3, 2] = 0.5, 0.5, 1.0
        return a, np.array([1.0, 2.0, 2.0, 1.0]) / 6.0
    if name == "dop853":
        from scipy.integrate._ivp import dop853_coefficients as d
        s = d.N_STAGES
        return np.array(d.A[:s, :s], dtype=np.float64), np.array(d.B, dtype=np.float64)
    raise ValueError(name)


def _segments(segs):
    arr = (Segment * len(segs))()
    for i, sg in enumerate(segs):
        M, steps, theta, rho = sg[:4]
        centre = sg[4] if len(sg) > 4 else 1
        arr[i] = Segment(int(M), int(steps), float(theta), float(rho), int(centre))
    return arr


def _tableau(tab):
    a, b = tab if not isinstance(tab, str) else tableau(tab)
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
    return Tableau(b.size, _p(a), _p(b)), (a, b)


def evolve_segments(prob: Problem, segs, tab, T: float, q0) -> np.ndarray:
    """segs: [(M, steps, theta, rho[, centre]), ...]; tab: 'rk4', 'dop853' or (a, b)."""
    sa = _segments(segs)
    tb, keep = _tableau(tab)
    q0 = _f64(q0)
    out = np.empty(2 * sa[len(segs) - 1].M)
    if lib().orc_evolve_segments(C.byref(prob), len(segs), sa, C.byref(tb), float(T), _p(q0), _p(out)) != 0:
        raise ValueError("invalid segments")
    return out


def shoot_segments(prob: Problem, segs, tab, c):
    sa = _segments(segs)
    tb, keep = _tableau(tab)
    c = _f64(c)
    M = sa[len(segs) - 1].M
    r, f = np.empty(M), np.empty(1)
    if lib().orc_shoot_segments(C.byref(prob), len(segs), sa, C.byref(tb), _p(c), _p(r), _p(f)) != 0:
        raise ValueError("invalid segments")
    return r, float(f[0])


def shoot_jacobian_segments(prob: Problem, segs, tab, c):
    """(r, J, f) on the last segment's grid; J is M_last x (n + 1), column 0 = d r / d T."""
    sa = _segments(segs)
    tb, keep = _tableau(tab)
    c = _f64(c)
    M = sa[len(segs) - 1].M
    r, f = np.empty(M), np.empty(1)
    Jc = np.empty((prob.n + 1, M))
    if lib().orc_shoot_jacobian_segments(C.byref(prob), len(segs), sa, C.byref(tb), _p(c), _p(r), _p(Jc),
                                         _p(f)) != 0:
        raise ValueError("invalid segments")
    return r, Jc.T.copy(), float(f[0])


def rhs_segment(prob: Problem, seg, T: float, y, ncol: int = 0, t_col: int = 0) -> np.ndarray:
    sa = _segments([seg])
    y = _f64(y).reshape(ncol + 1, 2 * sa[0].M)
    out = np.empty_like(y)
    lib().orc_rhs_segment(C.byref(prob), sa, float(T), _p(y), int(ncol), int(t_col), _p(out))
    return out


def dtn_segment(seg, h: float, eta, phi) -> np.ndarray:
    sa = _segments([seg])
    eta, phi = _f64(eta), _f64(phi)
    out = np.empty(eta.size)
    lib().orc_dtn_segment(sa, float(h), _p(eta), _p(phi), _p(out))
    return out


# ------------------------------------------------------------ the long double build
class WideProblem(C.Structure):
    _fields_ = [
        ("N", C.c_int), ("n", C.c_int), ("g", C.c_longdouble), ("tau", C.c_longdouble),
        ("h", C.c_longdouble), ("steps", C.c_int), ("basis", C.POINTER(C.c_longdouble)),
    ]


_L = C.POINTER(C.c_longdouble)
_wide = None


def wide_available() -> bool:
    """True where long double carries more precision than double."""
    return np.finfo(np.longdouble).eps < np.finfo(np.float64).eps


def wide_lib():
    global _wide
    with _lock:
        if _wide is None:
            L = C.CDLL(build(wide=True))
            P = C.POINTER(WideProblem)
            for name, (res, args) in {
                "orc_shoot": (None, [P, _L, _L, _L]),
                "orc_shoot_jacobian": (None, [P, _L, _L, _L, _L]),
                "orc_evolve": (None, [P, C.c_longdouble, _L, _L]),
                "orc_initial": (None, [P, _L, _L]),
                "orc_dtn": (None, [C.c_int, C.c_longdouble, _L, _L, C.c_int, _L]),
            }.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _wide = L
    return _wide


def _lp(a: np.ndarray):
    return a.ctypes.data_as(_L)


def _ld(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.longdouble))


def wide_problem(N, n, g=1.0, tau=0.0, h=1.0, steps=64, basis=None):
    """As make_problem, for the long double build (values converted exactly from double)."""
    keep = None
    bp = C.cast(None, _L)
    if basis is not None:
        keep = _ld(np.asarray(basis, dtype=np.float64).T)      # column k contiguous
        bp = _lp(keep)
    return WideProblem(int(N), int(n), g, tau, h, int(steps), bp), keep


def wide_shoot(prob: WideProblem, c):
    c = _ld(c)
    r, f = np.empty(prob.N, dtype=np.longdouble), np.empty(1, dtype=np.longdouble)
    wide_lib().orc_shoot(C.byref(prob), _lp(c), _lp(r), _lp(f))
    return r, f[0]


def wide_shoot_jacobian(prob: WideProblem, c):
    c = _ld(c)
    N, n = prob.N, prob.n
    r, f = np.empty(N, dtype=np.longdouble), np.empty(1, dtype=np.longdouble)
    Jc = np.empty((n + 1, N), dtype=np.longdouble)
    wide_lib().orc_shoot_jacobian(C.byref(prob), _lp(c), _lp(r), _lp(Jc), _lp(f))
    return r, Jc.T.copy(), f[0]


def wide_dtn(eta, phi, h) -> np.ndarray:
    eta, phi = _ld(eta), _ld(phi)
    out = np.empty(eta.size, dtype=np.longdouble)
    wide_lib().orc_dtn(eta.size, h, _lp(eta), _lp(phi), 1, _lp(out))
    return out


def objective_and_grad_segments(prob: Problem, segs, tab, c):
    """(f, grad) of the segmented shot by its discrete adjoint; grad[0] = d f / d T."""
    sa = _segments(segs)
    tb, keep = _tableau(tab)
    c = _f64(c)
    f, g = np.empty(1), np.empty(prob.n + 1)
    if lib().orc_objective_and_grad_segments(C.byref(prob), len(segs), sa, C.byref(tb), _p(c), _p(f),
                                             _p(g)) != 0:
        raise ValueError("invalid segments")
    return float(f[0]), g


def rhs_T_segment(prob: Problem, seg, q, kb):
    """(DF(q)^T kb, kb . F(q)) on a segment's mesh."""
    sa = _segments([seg])
    q, kb = _f64(q), _f64(kb)
    out, fd = np.empty_like(kb), np.empty(1)
    lib().orc_rhs_T_segment(C.byref(prob), sa, _p(q), _p(kb), _p(out), _p(fd))
    return out, float(fd[0])


def energy_segment(prob: Problem, seg, q) -> float:
    """The energy monitor of Sec. 4 for a state stored on a segment's mesh."""
    return lib().orc_energy_segment(C.byref(prob), _segments([seg]), _p(_f64(q)))
