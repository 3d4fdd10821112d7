"""Python binding of the BMPL C ABI (include/mpl.h).

Argument marshalling only: every step of the solve runs in the CUDA library
``_build/libmpl.so``.  The functions keep the C names (``mpl_create``,
``bmpl_solve``, ``mpl_destroy`` ...).  Arrays may be torch CUDA tensors (device
pointers are passed through) or C-contiguous numpy arrays (host pointers; the
library stages them through device memory).  There is no CPU fallback: if the
library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

# status codes (mpl_status_t)
MPL_OK = 0
MPL_ERR_ARG = 1
MPL_ERR_CUDA = 2
MPL_ERR_OOM = 3
MPL_ERR_TIMEOUT = 4
MPL_ERR_NOT_CONVERGED = 5
MPL_ERR_UNSUPPORTED = 6

# option keys (mpl_option_t)
MPL_OPT_RHO = 0
MPL_OPT_PRECISION = 1
MPL_OPT_MAX_OUTER = 2
MPL_OPT_SMAX = 3
MPL_OPT_EPS_IN = 4
MPL_OPT_INNER_MAX = 5
MPL_OPT_WARM_START = 6
MPL_OPT_SYNC_EVERY = 7
MPL_OPT_PROFILE = 8
MPL_OPT_GRAPH = 9
MPL_OPT_WARM_CANDIDATES = 10
MPL_OPT_WARM_MAX = 11
MPL_OPT_WARM_THRESHOLD = 12
MPL_OPT_QROUTE = 13
MPL_OPT_OMEGA = 14
MPL_OPT_STOP_RINF = 15
MPL_OPT_STOP_R2 = 16
MPL_OPT_STOP_EPS = 17
MPL_OPT_QGRAM = 18
MPL_OPT_GEMM_TILE = 19
MPL_OPT_REENTRY = 20
MPL_PROPOSAL_NPARAM = 4487

# limits of the allocation-free entry point (include/mpl.h)
MPL_NOALLOC_SCRATCH_BYTES = 1 << 20
MPL_NOALLOC_MAX_SIGNALS = (MPL_NOALLOC_SCRATCH_BYTES - 256) // 4

# per-signal status (mpl_signal_status_t)
MPL_SIG_CERTIFIED = 0
MPL_SIG_MAX_OUTER = 1
MPL_SIG_CAPACITY = 2
MPL_SIG_UNCERTIFIED = 3
MPL_SIG_NONFINITE = 4
MPL_SIG_EARLY_STOP = 5

EXPORTED = ("mpl_create", "bmpl_solve", "mpl_correlate", "mpl_destroy", "mpl_set_option", "mpl_get_option",
            "mpl_get_stats", "mpl_get_solution_f64", "mpl_get_phase_times", "mpl_get_launch_count",
            "mpl_status_string", "mpl_correlate_noalloc", "mpl_proposal_set_weights",
            "mpl_proposal_get_weights", "mpl_proposal_train", "mpl_proposal_loss_grad", "mpl_autotune")


class SignalStats(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int32), ("inner_iters", ctypes.c_int32),
                ("active_size", ctypes.c_int32), ("nnz", ctypes.c_int32), ("status", ctypes.c_int32),
                ("finishes", ctypes.c_int32), ("objective", ctypes.c_double), ("kkt", ctypes.c_double),
                ("gap", ctypes.c_double)]


class TuneResult(ctypes.Structure):
    _fields_ = [("qroute", ctypes.c_int32), ("sync_every", ctypes.c_int32), ("ms", ctypes.c_double),
                ("ms_default", ctypes.c_double), ("candidates", ctypes.c_int32), ("qgram", ctypes.c_int32),
                ("gemm_tile", ctypes.c_int32)]


class MplError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {mpl_status_string(code)} ({code})")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libmpl.so (building it first when it is absent or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library {_build.LIB} is missing; run paper_1302_5010_gb300.build.build()")
    lib = ctypes.CDLL(_build.LIB)
    vp, i32, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.mpl_create.argtypes = [vp, i32, i32, ctypes.POINTER(vp)]
    lib.mpl_create.restype = i32
    lib.bmpl_solve.argtypes = [vp, vp, i32, vp, vp, f64, vp]
    lib.bmpl_solve.restype = i32
    lib.mpl_correlate.argtypes = [vp, vp, i32, vp, vp]
    lib.mpl_correlate.restype = i32
    lib.mpl_correlate_noalloc.argtypes = [vp, i32, i32, vp, i32, vp, vp]
    lib.mpl_correlate_noalloc.restype = i32
    lib.mpl_proposal_set_weights.argtypes = [vp, vp, i32]
    lib.mpl_proposal_set_weights.restype = i32
    lib.mpl_proposal_get_weights.argtypes = [vp, vp, i32]
    lib.mpl_proposal_get_weights.restype = i32
    lib.mpl_proposal_train.argtypes = [vp, vp, i32, vp, vp, i32, f64, i32, ctypes.c_uint64, vp]
    lib.mpl_proposal_train.restype = i32
    lib.mpl_proposal_loss_grad.argtypes = [vp, vp, i32, vp, vp, ctypes.POINTER(f64), vp]
    lib.mpl_proposal_loss_grad.restype = i32
    lib.mpl_destroy.argtypes = [vp]
    lib.mpl_destroy.restype = None
    lib.mpl_set_option.argtypes = [vp, i32, f64]
    lib.mpl_set_option.restype = i32
    lib.mpl_get_option.argtypes = [vp, i32, ctypes.POINTER(f64)]
    lib.mpl_get_option.restype = i32
    lib.mpl_get_stats.argtypes = [vp, i32, ctypes.POINTER(SignalStats)]
    lib.mpl_get_stats.restype = i32
    lib.mpl_get_solution_f64.argtypes = [vp, i32, vp]
    lib.mpl_get_solution_f64.restype = i32
    lib.mpl_get_phase_times.argtypes = [vp, ctypes.POINTER(f64), i32]
    lib.mpl_get_phase_times.restype = i32
    lib.mpl_get_launch_count.argtypes = [vp]
    lib.mpl_get_launch_count.restype = ctypes.c_int64
    lib.mpl_autotune.argtypes = [vp, vp, i32, vp, f64, vp, ctypes.POINTER(TuneResult)]
    lib.mpl_autotune.restype = i32
    lib.mpl_status_string.argtypes = [i32]
    lib.mpl_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _ptr(a):
    """Raw pointer of a torch tensor (device or host) or a numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def mpl_status_string(code: int) -> str:
    return load().mpl_status_string(int(code)).decode()


def mpl_create(A, n: int, m: int):
    """A: atom-major (m, n) float32 (column-major n x m), device tensor or host array."""
    h = ctypes.c_void_p()
    rc = load().mpl_create(_ptr(A), int(n), int(m), ctypes.byref(h))
    if rc != MPL_OK:
        raise MplError(rc, "mpl_create")
    return h


def mpl_destroy(h) -> None:
    load().mpl_destroy(h)


def mpl_set_option(h, key: int, value: float) -> None:
    rc = load().mpl_set_option(h, int(key), float(value))
    if rc != MPL_OK:
        raise MplError(rc, f"mpl_set_option({key})")


def mpl_get_option(h, key: int) -> float:
    v = ctypes.c_double()
    rc = load().mpl_get_option(h, int(key), ctypes.byref(v))
    if rc != MPL_OK:
        raise MplError(rc, f"mpl_get_option({key})")
    return v.value


def bmpl_solve(h, B, p: int, lam, X, tol: float, stream=None) -> int:
    """Returns MPL_OK or MPL_ERR_NOT_CONVERGED; raises on any other status."""
    rc = load().bmpl_solve(h, _ptr(B), int(p), _ptr(lam), _ptr(X), float(tol), _stream_ptr(stream))
    if rc not in (MPL_OK, MPL_ERR_NOT_CONVERGED):
        raise MplError(rc, "bmpl_solve")
    return rc


def mpl_correlate(h, R, p: int, C, stream=None) -> None:
    """C (p, m) = rows of A^T R for R (p, n), by the handle's correlation path."""
    rc = load().mpl_correlate(h, _ptr(R), int(p), _ptr(C), _stream_ptr(stream))
    if rc != MPL_OK:
        raise MplError(rc, "mpl_correlate")


def mpl_correlate_noalloc(A, n: int, m: int, R, p: int, C, stream=None) -> int:
    """Allocation-free FP32 correlation (no handle): C (p, m) = rows of A^T R,
    all three device arrays.  Returns the status code (no exception), so that
    callers can see MPL_ERR_UNSUPPORTED / MPL_ERR_ARG."""
    return int(load().mpl_correlate_noalloc(_ptr(A), int(n), int(m), _ptr(R), int(p), _ptr(C),
                                            _stream_ptr(stream)))


def mpl_proposal_set_weights(h, w) -> None:
    w = np.ascontiguousarray(w, dtype=np.float32)
    rc = load().mpl_proposal_set_weights(h, _ptr(w), int(w.size))
    if rc != MPL_OK:
        raise MplError(rc, "mpl_proposal_set_weights")


def mpl_proposal_get_weights(h) -> np.ndarray:
    w = np.zeros(MPL_PROPOSAL_NPARAM, dtype=np.float32)
    rc = load().mpl_proposal_get_weights(h, _ptr(w), int(w.size))
    if rc != MPL_OK:
        raise MplError(rc, "mpl_proposal_get_weights")
    return w


def mpl_proposal_train(h, B, p: int, lam, Xref, epochs: int, lr: float, batch: int, seed: int) -> np.ndarray:
    losses = np.zeros(max(epochs, 1), dtype=np.float32)
    rc = load().mpl_proposal_train(h, _ptr(B), int(p), _ptr(lam), _ptr(Xref), int(epochs), float(lr), int(batch),
                                   ctypes.c_uint64(seed), _ptr(losses))
    if rc != MPL_OK:
        raise MplError(rc, "mpl_proposal_train")
    return losses[:epochs]


def mpl_proposal_loss_grad(h, B, p: int, lam, Xref):
    g = np.zeros(MPL_PROPOSAL_NPARAM, dtype=np.float32)
    loss = ctypes.c_double()
    rc = load().mpl_proposal_loss_grad(h, _ptr(B), int(p), _ptr(lam), _ptr(Xref), ctypes.byref(loss), _ptr(g))
    if rc != MPL_OK:
        raise MplError(rc, "mpl_proposal_loss_grad")
    return loss.value, g


def mpl_get_stats(h, p: int) -> dict:
    arr = (SignalStats * max(p, 1))()
    rc = load().mpl_get_stats(h, int(p), arr)
    if rc != MPL_OK:
        raise MplError(rc, "mpl_get_stats")
    return {f: np.array([getattr(arr[i], f) for i in range(p)]) for f, _ in SignalStats._fields_}


def mpl_get_solution_f64(h, p: int, X64) -> None:
    rc = load().mpl_get_solution_f64(h, int(p), _ptr(X64))
    if rc != MPL_OK:
        raise MplError(rc, "mpl_get_solution_f64")


def mpl_get_phase_times(h) -> list:
    buf = (ctypes.c_double * 16)()
    k = load().mpl_get_phase_times(h, buf, 16)
    return [buf[i] for i in range(k)]


def mpl_autotune(h, B, p: int, lam, tol: float, stream=None) -> dict:
    """Time the candidate settings on this batch and keep the fastest (include/mpl.h)."""
    out = TuneResult()
    rc = load().mpl_autotune(h, _ptr(B), int(p), _ptr(lam), float(tol), _stream_ptr(stream), ctypes.byref(out))
    if rc != MPL_OK:
        raise MplError(rc, "mpl_autotune")
    return {f: getattr(out, f) for f, _ in TuneResult._fields_}


def mpl_get_launch_count(h) -> int:
    return int(load().mpl_get_launch_count(h))


PHASES = ("total", "correlation", "selection", "gram", "finish", "master", "residual", "corr_columns",
          "finish_flops", "qroute_columns", "qroute", "apg_elems", "apg_global_elems", "residual_bytes",
          "gram_bytes", "finish_bytes")


@dataclass
class SolveResult:
    status: int
    stats: dict


class Solver:
    """Owns one handle.  ``solve`` takes torch CUDA tensors (B (p, n), lam (p,),
    X (p, m)) or numpy arrays and runs bmpl_solve on the current stream."""

    def __init__(self, At, rho: int = 1, precision: int = 0, **opts):
        m, n = At.shape
        self.n, self.m = int(n), int(m)
        self.h = mpl_create(At, self.n, self.m)
        mpl_set_option(self.h, MPL_OPT_RHO, rho)
        mpl_set_option(self.h, MPL_OPT_PRECISION, precision)
        keys = dict(max_outer=MPL_OPT_MAX_OUTER, smax=MPL_OPT_SMAX, eps_in=MPL_OPT_EPS_IN,
                    inner_max=MPL_OPT_INNER_MAX, warm_start=MPL_OPT_WARM_START, profile=MPL_OPT_PROFILE,
                    sync_every=MPL_OPT_SYNC_EVERY, graph=MPL_OPT_GRAPH, warm_candidates=MPL_OPT_WARM_CANDIDATES,
                    warm_max=MPL_OPT_WARM_MAX, warm_threshold=MPL_OPT_WARM_THRESHOLD, qroute=MPL_OPT_QROUTE,
                    omega=MPL_OPT_OMEGA, stop_rinf=MPL_OPT_STOP_RINF, stop_r2=MPL_OPT_STOP_R2,
                    stop_eps=MPL_OPT_STOP_EPS, qgram=MPL_OPT_QGRAM, gemm_tile=MPL_OPT_GEMM_TILE,
                    reentry=MPL_OPT_REENTRY)
        for k, v in opts.items():
            mpl_set_option(self.h, keys[k], v)

    def set(self, key: int, value: float) -> None:
        mpl_set_option(self.h, key, value)

    def get(self, key: int) -> float:
        return mpl_get_option(self.h, key)

    def solve(self, B, lam, X, tol: float = 1e-6, stream=None) -> SolveResult:
        p = B.shape[0]
        rc = bmpl_solve(self.h, B, p, lam, X, tol, stream)
        return SolveResult(rc, mpl_get_stats(self.h, p))

    def train_proposal(self, B, lam, Xref, epochs: int = 4, lr: float = 3e-3, batch: int = 2048,
                       seed: int = 9000) -> np.ndarray:
        """Train the warm-start proposal on signals B (p, n) with reference solutions
        Xref (p, m); returns the mean loss per epoch."""
        return mpl_proposal_train(self.h, B, B.shape[0], lam, Xref, epochs, lr, batch, seed)

    def autotune(self, B, lam, tol: float = 1e-6, stream=None) -> dict:
        return mpl_autotune(self.h, B, B.shape[0], lam, tol, stream)

    def correlate(self, R, C, stream=None) -> None:
        mpl_correlate(self.h, R, R.shape[0], C, stream)

    def solution_f64(self, X64) -> None:
        mpl_get_solution_f64(self.h, X64.shape[0], X64)

    def phase_times(self) -> dict:
        return dict(zip(PHASES, mpl_get_phase_times(self.h)))

    def launches(self) -> int:
        return mpl_get_launch_count(self.h)

    def close(self) -> None:
        if self.h is not None:
            mpl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
