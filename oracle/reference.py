"""ctypes wrappers of the plain-C oracle (``cqk_oracle.c``).  Test infrastructure.

The shared library is compiled on first use with gcc (-O2 -ffp-contract=off,
no fast-math) into ``oracle/_build/``; ``__graft_entry__.build()`` compiles it
too.  All arrays are float64, C-contiguous numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cqk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libcqk_oracle.so")
_lock = threading.Lock()
_lib = None

# machine epsilon^{3/4} of the stopping criteria of Sec. 4
EPS34_F64 = float(np.finfo(np.float64).eps) ** 0.75
EPS34_F32 = float(np.finfo(np.float32).eps) ** 0.75

STOP_NAMES = {0: "none", 1: "exact", 2: "residual", 3: "step", 4: "same", 5: "bracket", 6: "below"}
_STATUS = {0: "ok", 1: "infeasible", 2: "maxiter", 3: "bad_input"}


def build(force: bool = False) -> str:
    """Compile cqk_oracle.c into a shared library (idempotent)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _SO + f".{os.getpid()}.tmp"
            subprocess.check_call(
                ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
                 "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        # CQK_ORACLE_SO lets the mutation tests load a deliberately broken copy
        path = os.environ.get("CQK_ORACLE_SO") or build()
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        d_p, i64_p, i_p = P(ctypes.c_double), P(ctypes.c_int64), P(ctypes.c_int)
        i64, dbl, cint = ctypes.c_int64, ctypes.c_double, ctypes.c_int
        lib.cqko_x.argtypes = [i64, d_p, d_p, d_p, d_p, d_p, dbl, d_p]
        lib.cqko_phi.argtypes = [i64, d_p, d_p, d_p, d_p, d_p, dbl, d_p]
        lib.cqko_lambda0.argtypes = [i64, d_p, d_p, d_p, dbl]
        lib.cqko_lambda0.restype = dbl
        lib.cqko_breakpoint.argtypes = [i64, d_p, d_p, d_p, d_p, d_p, dbl, cint, i_p]
        lib.cqko_breakpoint.restype = dbl
        lib.cqko_newton.argtypes = [i64, d_p, d_p, d_p, d_p, d_p, dbl, dbl, cint, dbl,
                                    d_p, i_p, i_p, i_p, i_p, d_p, d_p]
        lib.cqko_newton.restype = cint
        lib.cqko_solve_sort.argtypes = [i64, d_p, d_p, d_p, d_p, d_p, dbl, d_p, d_p]
        lib.cqko_solve_sort.restype = cint
        lib.cqko_condat_init.argtypes = [d_p, i64_p, i64, dbl, cint, d_p, i64_p, i64_p, d_p]
        lib.cqko_condat_init.restype = dbl
        lib.cqko_condat_chunks.argtypes = [i64, d_p, dbl, cint, i64, i64, i64, d_p, i64_p]
        lib.cqko_condat_chunks.restype = dbl
        lib.cqko_condat_chunks_warm.argtypes = [i64, d_p, d_p, dbl, cint, i64, i64, i64, d_p, i64_p]
        lib.cqko_condat_chunks_warm.restype = dbl
        lib.cqko_lambda0_warm.argtypes = [i64, d_p, d_p, d_p, d_p, d_p, d_p, dbl]
        lib.cqko_lambda0_warm.restype = dbl
        lib.cqko_condat.argtypes = [i64, d_p, dbl, d_p]
        lib.cqko_condat.restype = dbl
        lib.cqko_newton_simplex.argtypes = [i64, d_p, dbl, cint, dbl, cint, dbl, d_p, i_p, i_p, d_p]
        lib.cqko_newton_simplex.restype = cint
        lib.cqko_project_simplex_sort.argtypes = [i64, d_p, dbl, d_p]
        lib.cqko_project_simplex_sort.restype = dbl
        _lib = lib
    return _lib


def set_threads(t: int) -> int:
    """Threads of the oracle's loops over all variables; 1 (the default) is the plain sequential
    oracle.  More threads run the same algorithms with OpenMP-parallel map-reduce passes (the
    paper's CPU Jacobi form), for the all-core CPU baseline only.  Returns the previous value."""
    lib = _load()
    lib.cqko_set_threads.argtypes = [ctypes.c_int]
    lib.cqko_get_threads.restype = ctypes.c_int
    prev = int(lib.cqko_get_threads())
    lib.cqko_set_threads(int(t))
    return prev


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _ptr(x):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _arrs(a, b, d, l, u):
    a, b, d, l, u = (_f64(v) for v in (a, b, d, l, u))
    n = a.shape[0]
    assert all(v.shape == (n,) for v in (b, d, l, u))
    return n, a, b, d, l, u


def x_of_lambda(lam, a, b, d, l, u):
    """eq. (xopt): x_i(lambda) = clip((b_i lambda + a_i)/d_i, l_i, u_i)."""
    n, a, b, d, l, u = _arrs(a, b, d, l, u)
    x = np.empty(n)
    _load().cqko_x(n, _ptr(a), _ptr(b), _ptr(d), _ptr(l), _ptr(u), float(lam), _ptr(x))
    return x


def phi(lam, a, b, d, l, u):
    """eq. (opt), eq. (phideriv): returns (phi, phi'_+, phi'_-, sum |b_i x_i|)."""
    n, a, b, d, l, u = _arrs(a, b, d, l, u)
    out = np.empty(4)
    _load().cqko_phi(n, _ptr(a), _ptr(b), _ptr(d), _ptr(l), _ptr(u), float(lam), _ptr(out))
    return tuple(float(v) for v in out)


def lambda0_formula(a, b, d, r):
    """eq. (CQKlambda0) with J = all variables."""
    a, b, d = _f64(a), _f64(b), _f64(d)
    return float(_load().cqko_lambda0(a.shape[0], _ptr(a), _ptr(b), _ptr(d), float(r)))


def lambda0_warm(a, b, d, l, u, xbar, r):
    """eq. (CQKlambda0) with J = {l < xbar < u} (all variables if that set is empty)."""
    n, a, b, d, l, u = _arrs(a, b, d, l, u)
    xbar = _f64(xbar)
    return float(_load().cqko_lambda0_warm(n, _ptr(a), _ptr(b), _ptr(d), _ptr(l), _ptr(u), _ptr(xbar),
                                           float(r)))


def breakpoint_search(lam, direction, a, b, d, l, u):
    """Closest finite breakpoint strictly right (direction>0) or left of lam; None if none."""
    n, a, b, d, l, u = _arrs(a, b, d, l, u)
    found = ctypes.c_int(0)
    v = _load().cqko_breakpoint(n, _ptr(a), _ptr(b), _ptr(d), _ptr(l), _ptr(u), float(lam),
                                1 if direction > 0 else -1, ctypes.byref(found))
    return float(v) if found.value else None


def newton_cqk(a, b, d, l, u, r, lam0=None, max_iter=100, eps34=EPS34_F64):
    """Alg. 1 with the stopping tests of Sec. 4.  lam0 defaults to eq. (CQKlambda0).

    Returns a dict: status, lam, x, evals (phi evaluations), bpsearch, stop,
    step (Newton step available at the stop, 0 if none), trace (lambda_k's).
    """
    n, a, b, d, l, u = _arrs(a, b, d, l, u)
    if lam0 is None:
        lam0 = lambda0_formula(a, b, d, r)
    lam = ctypes.c_double()
    ev, bp, ns, st = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    step = ctypes.c_double()
    trace = np.full(max_iter, np.nan)
    status = _load().cqko_newton(n, _ptr(a), _ptr(b), _ptr(d), _ptr(l), _ptr(u), float(r),
                                 float(lam0), int(max_iter), float(eps34), ctypes.byref(lam),
                                 ctypes.byref(ev), ctypes.byref(bp), ctypes.byref(ns),
                                 ctypes.byref(st), ctypes.byref(step), _ptr(trace))
    out = dict(status=_STATUS[status], lam=lam.value, evals=ev.value, bpsearch=bp.value,
               secant=ns.value, stop=STOP_NAMES[st.value], step=step.value,
               trace=trace[:ev.value].copy(), lam0=float(lam0))
    out["x"] = x_of_lambda(lam.value, a, b, d, l, u) if status == 0 else None
    return out


def solve_sort(a, b, d, l, u, r):
    """Exact solution by sorting the breakpoints.  Returns (status, lam*, x*)."""
    n, a, b, d, l, u = _arrs(a, b, d, l, u)
    lam = ctypes.c_double()
    x = np.empty(n)
    st = _load().cqko_solve_sort(n, _ptr(a), _ptr(b), _ptr(d), _ptr(l), _ptr(u), float(r),
                                 ctypes.byref(lam), _ptr(x))
    if st != 0:
        return _STATUS[st], None, None
    return "ok", lam.value, x


def condat_init(y, r, idx=None, l1=False, return_trace=False):
    """Alg. 2 on the ordered subset idx (default: all).  Returns (lambda_J, sum_J y, |J|)
    and, with return_trace, the multiplier after each entry of the first loop."""
    y = _f64(y)
    idx = np.arange(y.shape[0], dtype=np.int64) if idx is None else np.ascontiguousarray(idx, dtype=np.int64)
    p = idx.shape[0]
    scratch = np.empty(max(2 * p, 2), dtype=np.int64)
    trace = np.full(max(p, 1), np.nan)
    js = ctypes.c_double()
    jc = ctypes.c_int64()
    lam = _load().cqko_condat_init(_ptr(y), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), p,
                                   float(r), 1 if l1 else 0, ctypes.byref(js), ctypes.byref(jc),
                                   scratch.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(trace))
    if return_trace:
        return float(lam), js.value, jc.value, trace[:p].copy()
    return float(lam), js.value, jc.value


def condat_chunks(y, r, tile, nchunks, l1=False, shift=0):
    """Parallel lambda_0 of Sec. 4 over the partition chunk(i) = ((i + shift) // tile) % nchunks.

    Returns (lambda_0, sum over the union of J's, size of the union)."""
    y = _f64(y)
    us = ctypes.c_double()
    uc = ctypes.c_int64()
    lam = _load().cqko_condat_chunks(y.shape[0], _ptr(y), float(r), 1 if l1 else 0, int(tile),
                                     int(nchunks), int(shift), ctypes.byref(us), ctypes.byref(uc))
    return float(lam), us.value, uc.value


def condat_chunks_warm(y, xbar, r, tile, nchunks, l1=False, shift=0):
    """Warm start of Sec. 3.3 over the chunk partition: Alg. 2 per chunk on supp(xbar).
    Returns (lambda_0, sum over the union of J's, size of the union)."""
    y, xbar = _f64(y), _f64(xbar)
    us = ctypes.c_double()
    uc = ctypes.c_int64()
    lam = _load().cqko_condat_chunks_warm(y.shape[0], _ptr(y), _ptr(xbar), float(r), 1 if l1 else 0, int(tile),
                                          int(nchunks), int(shift), ctypes.byref(us), ctypes.byref(uc))
    return float(lam), us.value, uc.value


def condat_project(y, r):
    """Alg. 3: Condat's projection onto {x >= 0, sum x = r}.  Returns (lam, x)."""
    y = _f64(y)
    x = np.empty_like(y)
    lam = _load().cqko_condat(y.shape[0], _ptr(y), float(r), _ptr(x))
    return float(lam), x


def newton_simplex(y, r, lam0=None, l1=False, max_iter=100, eps34=EPS34_F64):
    """Alg. 4 on y (|y| when l1) from lam0 (default: eq. (CQKlambda0) specialised,
    (r - sum y)/n).  Returns dict(status, lam, x (of the simplex problem), evals, stop, trace)."""
    y = _f64(y)
    n = y.shape[0]
    yy = np.abs(y) if l1 else y
    if lam0 is None:
        lam0 = (r - float(np.sum(yy, dtype=np.longdouble))) / n
    lam = ctypes.c_double()
    ev, st = ctypes.c_int(), ctypes.c_int()
    trace = np.full(max_iter, np.nan)
    status = _load().cqko_newton_simplex(n, _ptr(y), float(r), 1 if l1 else 0, float(lam0),
                                         int(max_iter), float(eps34), ctypes.byref(lam),
                                         ctypes.byref(ev), ctypes.byref(st), _ptr(trace))
    x = np.maximum(0.0, yy + lam.value)
    return dict(status=_STATUS[status], lam=lam.value, x=x, evals=ev.value,
                stop=STOP_NAMES[st.value], trace=trace[:ev.value].copy(), lam0=float(lam0))


def project_simplex_sort(y, r):
    """Sort-based projection onto {x >= 0, sum x = r}.  Returns (lam*, x*)."""
    y = _f64(y)
    x = np.empty_like(y)
    lam = _load().cqko_project_simplex_sort(y.shape[0], _ptr(y), float(r), _ptr(x))
    return float(lam), x
