"""FP64 CPU oracle for MPL/BMPL -- test infrastructure.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The CUDA library never calls it, and it shares
no code with the CUDA path.  ``mpl_oracle.c`` follows Algorithm 1 of the paper
(with an exact sign-fixed finish of every master problem), ``checkers.py``
holds independent algorithms (coordinate descent, brute force, closed forms)
that pin it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class Opts(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_int), ("max_outer", ctypes.c_int), ("s_max", ctypes.c_int),
                ("max_attempts", ctypes.c_int), ("exact_finish", ctypes.c_int),
                ("corr_route", ctypes.c_int), ("eps_in", ctypes.c_double), ("omega", ctypes.c_int),
                ("stop_rinf", ctypes.c_double), ("stop_r2", ctypes.c_double), ("stop_eps", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("n_outer", ctypes.c_int), ("n_inner", ctypes.c_int), ("S_size", ctypes.c_int),
                ("status", ctypes.c_int), ("nnz", ctypes.c_int), ("objective", ctypes.c_double),
                ("kkt", ctypes.c_double), ("gap", ctypes.c_double)]


class Trace(ctypes.Structure):
    _fields_ = [("cap", ctypes.c_int), ("rho_cap", ctypes.c_int),
                ("n_added", ctypes.POINTER(ctypes.c_int)), ("added", ctypes.POINTER(ctypes.c_int)),
                ("gsel", ctypes.POINTER(ctypes.c_double)), ("f_prev", ctypes.POINTER(ctypes.c_double)),
                ("f_first", ctypes.POINTER(ctypes.c_double)), ("L_first", ctypes.POINTER(ctypes.c_double)),
                ("f_iter", ctypes.POINTER(ctypes.c_double)), ("inner", ctypes.POINTER(ctypes.c_int))]


def build(force: bool = False) -> str:
    """Compile mpl_oracle.c with gcc (plain -O2, OpenMP across signals only)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_mpl.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                   ctypes.POINTER(Opts), dp, ctypes.POINTER(Result), ctypes.POINTER(Trace)]
        lib.oracle_mpl.restype = ctypes.c_int
        lib.oracle_bmpl.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp,
                                    ctypes.POINTER(Opts), ctypes.c_int, dp, ctypes.POINTER(Result)]
        lib.oracle_bmpl.restype = ctypes.c_int
        lib.oracle_certify.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, dp,
                                       dp, dp, dp, ctypes.POINTER(ctypes.c_int)]
        lib.oracle_certify.restype = ctypes.c_int
        lib.oracle_default_opts.argtypes = [ctypes.POINTER(Opts)]
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _opts(rho: int, **kw) -> Opts:
    o = Opts()
    _load().oracle_default_opts(ctypes.byref(o))
    o.rho = int(rho)
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown oracle option {k}")
        setattr(o, k, type(getattr(o, k))(v))
    return o


def _res_dict(r: Result) -> dict:
    return {f: getattr(r, f) for f, _ in Result._fields_}


def mpl(At, b, lam: float, rho: int, trace_cap: int = 256, **opts):
    """Algorithm 1 on one signal.  At: (m, n) atom-major, b: (n,).
    Returns (x, result, trace)."""
    A = np.ascontiguousarray(At, dtype=np.float64)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    m, n = A.shape
    o = _opts(rho, **opts)
    x = np.zeros(m, dtype=np.float64)
    res = Result()
    rc_ = max(1, int(rho))
    arrs = dict(n_added=np.zeros(trace_cap, np.int32), added=np.full(trace_cap * rc_, -1, np.int32),
                gsel=np.zeros(trace_cap * rc_), f_prev=np.zeros(trace_cap), f_first=np.zeros(trace_cap),
                L_first=np.zeros(trace_cap), f_iter=np.zeros(trace_cap), inner=np.zeros(trace_cap, np.int32))
    tr = Trace()
    tr.cap, tr.rho_cap = trace_cap, rc_
    for k, v in arrs.items():
        ct = ctypes.c_int if v.dtype == np.int32 else ctypes.c_double
        setattr(tr, k, v.ctypes.data_as(ctypes.POINTER(ct)))
    rc = _load().oracle_mpl(_dptr(A), n, m, _dptr(bb), float(lam), ctypes.byref(o), _dptr(x),
                            ctypes.byref(res), ctypes.byref(tr))
    if rc != 0:
        raise RuntimeError(f"oracle_mpl failed ({rc})")
    r = _res_dict(res)
    T = min(r["n_outer"], trace_cap)
    trace = dict(n_added=arrs["n_added"][:T].copy(),
                 added=[arrs["added"][t * rc_: t * rc_ + arrs["n_added"][t]].copy() for t in range(T)],
                 gsel=[arrs["gsel"][t * rc_: t * rc_ + arrs["n_added"][t]].copy() for t in range(T)],
                 f_prev=arrs["f_prev"][:T].copy(), f_first=arrs["f_first"][:T].copy(),
                 L_first=arrs["L_first"][:T].copy(), f_iter=arrs["f_iter"][:T].copy(),
                 inner=arrs["inner"][:T].copy())
    return x, r, trace


def bmpl(At, B, lam, rho: int, threads: int = 0, **opts):
    """Batch mode over the rows of B (p, n).  Returns (X (p, m), results dict of arrays)."""
    A = np.ascontiguousarray(At, dtype=np.float64)
    Bd = np.ascontiguousarray(B, dtype=np.float64)
    lm = np.ascontiguousarray(lam, dtype=np.float64).reshape(-1)
    m, n = A.shape
    p = Bd.shape[0]
    o = _opts(rho, **opts)
    X = np.zeros((p, m), dtype=np.float64)
    res = (Result * max(p, 1))()
    rc = _load().oracle_bmpl(_dptr(A), n, m, _dptr(Bd), p, _dptr(lm), ctypes.byref(o), int(threads),
                             _dptr(X), res)
    if rc != 0:
        raise RuntimeError(f"oracle_bmpl failed ({rc})")
    out = {f: np.array([getattr(res[i], f) for i in range(p)]) for f, _ in Result._fields_}
    return X, out


def certify(At, b, lam: float, x) -> dict:
    """Objective, KKT violation / lambda and relative duality gap of x, in FP64."""
    A = np.ascontiguousarray(At, dtype=np.float64)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    m, n = A.shape
    obj, kkt, gap = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    nnz = ctypes.c_int()
    rc = _load().oracle_certify(_dptr(A), n, m, _dptr(bb), float(lam), _dptr(xx), ctypes.byref(obj),
                                ctypes.byref(kkt), ctypes.byref(gap), ctypes.byref(nnz))
    if rc != 0:
        raise RuntimeError("oracle_certify failed")
    return dict(objective=obj.value, kkt=kkt.value, gap=gap.value, nnz=nnz.value)


def num_threads() -> int:
    return int(_load().oracle_num_threads())
