"""Shared parity checks between the CUDA path and the FP64 oracle.

Tolerances are the acceptance numbers of the method's GPU/oracle comparison:
relative objective difference <= 1e-6, ||X - X_o||_F / ||X_o||_F <= 1e-4, and
identical supports for coefficients above 1e-3 * max|x|.
"""
import numpy as np

OBJ_RTOL = 1e-6
X_RTOL = 1e-4
SUPP_FRAC = 1e-3


def objective(At64, b, x, lam):
    r = b - At64.T @ x
    return lam * np.abs(x).sum() + 0.5 * r @ r


def check_against_oracle(P, X_gpu, X_or, idx=None):
    """X_gpu, X_or: (p', m) for the signals idx (default all)."""
    idx = np.arange(P.p) if idx is None else np.asarray(idx)
    A64 = P.At.astype(np.float64)
    X_gpu = np.asarray(X_gpu, dtype=np.float64)
    X_or = np.asarray(X_or, dtype=np.float64)
    num = np.linalg.norm(X_gpu - X_or)
    den = np.linalg.norm(X_or)
    if den > 0:
        assert num / den <= X_RTOL, f"||X-Xo||/||Xo|| = {num / den:.3e}"
    else:
        assert num == 0.0
    for row, i in enumerate(idx):
        b = P.B[i].astype(np.float64)
        lam = float(P.lam[i])
        fg = objective(A64, b, X_gpu[row], lam)
        fo = objective(A64, b, X_or[row], lam)
        assert abs(fg - fo) <= OBJ_RTOL * abs(fo), f"signal {i}: objective {fg} vs {fo}"
        xm = np.abs(X_or[row]).max()
        if xm > 0:
            sg = np.abs(X_gpu[row]) > SUPP_FRAC * xm
            so = np.abs(X_or[row]) > SUPP_FRAC * xm
            assert np.array_equal(sg, so), f"signal {i}: supports differ at {np.nonzero(sg ^ so)[0]}"
        else:
            assert np.all(X_gpu[row] == 0)
