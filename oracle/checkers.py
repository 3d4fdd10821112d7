"""Independent LASSO solvers and certificates that pin the MPL oracle.

Test infrastructure.  None of these functions shares code with
``mpl_oracle.c``; each reaches the LASSO minimiser of eq. 2,
    min_x lambda*||x||_1 + 0.5*||b - A x||^2,
by a different route, so a dropped term, a wrong sign or a transposed operand
in the oracle shows up as a disagreement:

  * ``soft_threshold_orthonormal``: closed form when A^T A = I;
  * ``bruteforce_lasso``: enumerate every sign pattern of a tiny problem and
    keep the best point satisfying the on-support optimality system;
  * ``cd_lasso``: cyclic coordinate descent (the method the paper cites among
    the l1 solvers of Sec. 1);
  * ``omp``: orthogonal matching pursuit, which MPL reduces to for lambda = 0
    and rho = 1 (Sec. 2.3);
  * ``kkt_violation`` / ``duality_gap``: the optimality conditions of eq. 2
    and the scaled dual point of eq. 5.

Layouts as in ``paper_1302_5010_gb300.synth``: At is (m, n) atom-major.
"""
from __future__ import annotations

import itertools

import numpy as np


def objective(At, b, x, lam) -> float:
    A = np.asarray(At, dtype=np.float64)
    r = np.asarray(b, dtype=np.float64) - A.T @ np.asarray(x, dtype=np.float64)
    return float(lam * np.abs(x).sum() + 0.5 * r @ r)


def kkt_violation(At, b, x, lam) -> float:
    """max_j of |a_j^T r - lambda*sign(x_j)| on the support and
    (|a_j^T r| - lambda)_+ off it, divided by lambda."""
    A = np.asarray(At, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    r = np.asarray(b, dtype=np.float64) - A.T @ x
    g = A @ r
    on = x != 0
    v_on = np.abs(g[on] - lam * np.sign(x[on]))
    v_off = np.maximum(np.abs(g[~on]) - lam, 0.0)
    worst = max(v_on.max(initial=0.0), v_off.max(initial=0.0))
    return float(worst / lam) if lam > 0 else float(worst)


def duality_gap(At, b, x, lam) -> float:
    """(P(x) - D(alpha)) / P(x) with alpha = r * min(1, lambda/||A^T r||_inf),
    a feasible point of the dual eq. 5 (tau = all ones)."""
    A = np.asarray(At, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    r = b - A.T @ x
    P = lam * np.abs(x).sum() + 0.5 * r @ r
    ginf = np.abs(A @ r).max()
    alpha = r * (min(1.0, lam / ginf) if ginf > 0 else 1.0)
    D = -0.5 * alpha @ alpha + alpha @ b
    return float((P - D) / P) if P > 0 else 0.0


def soft_threshold_orthonormal(At, b, lam):
    """Closed-form minimiser when A^T A = I: x = soft(A^T b, lambda)."""
    g = np.asarray(At, dtype=np.float64) @ np.asarray(b, dtype=np.float64)
    return np.sign(g) * np.maximum(np.abs(g) - lam, 0.0)


def bruteforce_lasso(At, b, lam):
    """Exact minimiser for tiny m (3^m sign patterns).  For each pattern s the
    stationarity of eq. 2 on P = supp(s) reads A_P^T A_P z = A_P^T b - lam*s_P;
    a solution whose signs agree with s is a candidate, and the smallest
    objective among candidates (and x = 0) is the minimiser."""
    A = np.asarray(At, dtype=np.float64).T  # n x m
    b = np.asarray(b, dtype=np.float64)
    n, m = A.shape
    best_x = np.zeros(m)
    best_f = 0.5 * b @ b
    for pattern in itertools.product((-1, 0, 1), repeat=m):
        s = np.array(pattern, dtype=np.float64)
        P = np.nonzero(s)[0]
        if len(P) == 0 or len(P) > n:
            continue
        AP = A[:, P]
        M = AP.T @ AP
        try:
            z = np.linalg.solve(M, AP.T @ b - lam * s[P])
        except np.linalg.LinAlgError:
            continue
        if np.all(z * s[P] > 0):
            x = np.zeros(m)
            x[P] = z
            r = b - A @ x
            f = lam * np.abs(x).sum() + 0.5 * r @ r
            if f < best_f:
                best_f, best_x = f, x
    return best_x


def cd_lasso(At, b, lam, tol=1e-14, max_sweeps=200000):
    """Cyclic coordinate descent: x_j <- soft(x_j*|a_j|^2 + a_j^T r, lam)/|a_j|^2,
    sweeping the current support until it settles, then a full sweep to check."""
    A = np.asarray(At, dtype=np.float64)  # m x n
    b = np.asarray(b, dtype=np.float64)
    m, n = A.shape
    nrm2 = np.einsum("ij,ij->i", A, A)
    x = np.zeros(m)
    r = b.copy()

    def sweep(idx):
        dmax = 0.0
        for j in idx:
            if nrm2[j] == 0:
                continue
            rho_j = A[j] @ r + x[j] * nrm2[j]
            new = np.sign(rho_j) * max(abs(rho_j) - lam, 0.0) / nrm2[j]
            d = new - x[j]
            if d != 0.0:
                r[:] -= d * A[j]
                x[j] = new
                dmax = max(dmax, abs(d))
        return dmax

    for _ in range(max_sweeps):
        dfull = sweep(range(m))
        if dfull <= tol:
            break
        act = np.nonzero(x)[0]
        for _ in range(max_sweeps):
            if sweep(act) <= tol:
                break
    return x


def omp(At, b, k):
    """Orthogonal matching pursuit for k steps (argmax |a_j^T r| outside the
    support, lower index on ties; least squares on the support).
    Returns (x, list of selected indices in order)."""
    A = np.asarray(At, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m, n = A.shape
    S = []
    r = b.copy()
    z = np.zeros(0)
    for _ in range(k):
        g = np.abs(A @ r)
        g[S] = -1.0
        j = int(np.argmax(g))  # first maximum = lowest index on ties
        S.append(j)
        z, *_ = np.linalg.lstsq(A[S].T, b, rcond=None)
        r = b - A[S].T @ z
    x = np.zeros(m)
    x[S] = z
    return x, S
