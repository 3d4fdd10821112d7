"""Early stopping (Sec. 2.5, eqs. stop1 and stop_con) and the lambda = 0 path
(least squares; with rho = 1 the OMP reduction of Sec. 2.5) on the GPU.

A stopped signal returns the exact minimiser of eq. 2 restricted to its final
active set; the rules are tested on the GPU's own iterates, which are FP32
master-problem solutions, so the iteration at which a rule fires can differ
from the oracle's exact iterates near a threshold.  The tests therefore check
what holds for any correct implementation: the rule holds at the returned
point, the point is optimal on its support, the run stops no later than the
full solve, and, where the paths cannot differ, equality with the oracle."""
import numpy as np
import pytest

import oracle
from oracle import checkers as ck
from paper_1302_5010_gb300 import mpl, synth
from parity import check_against_oracle
from test_gpu_parity import solve_gpu

pytestmark = pytest.mark.gpu


def _restricted_kkt(At, b, lam, x):
    """max over supp(x) of |a_j^T r - lambda sign(x_j)| (FP64)."""
    A = At.astype(np.float64)
    r = b.astype(np.float64) - A.T @ x
    g = A @ r
    S = np.flatnonzero(x)
    return np.max(np.abs(g[S] - lam * np.sign(x[S]))) if S.size else 0.0, g


def test_residual_rule_above_norm_returns_zero():
    P = synth.small_problem(128, 512, 6, 4, 8, rho=3, seed=21)
    X, X64, res = solve_gpu(P, stop_r2=1e9)
    assert res.status == mpl.MPL_OK
    assert np.all(res.stats["status"] == mpl.MPL_SIG_EARLY_STOP)
    assert not np.any(X64)
    for i in range(P.p):  # the oracle stops at its first check as well
        x, r, _ = oracle.mpl(P.At, P.B[i], P.lam[i], P.rho, stop_r2=1e9)
        assert r["status"] == 3 and not np.any(x)


def test_correlation_rule():
    P = synth.small_problem(256, 1024, 12, 10, 30, rho=4, seed=22, lam_frac=0.01)
    Xf, X64f, rf = solve_gpu(P)
    rinf = 3.0 * P.lam  # per signal would be ideal; the option is global: use the median scale
    R = float(np.median(rinf))
    X, X64, res = solve_gpu(P, stop_rinf=R)
    st = res.stats
    assert np.all((st["status"] == mpl.MPL_SIG_EARLY_STOP) | (st["status"] == mpl.MPL_SIG_CERTIFIED))
    assert np.any(st["status"] == mpl.MPL_SIG_EARLY_STOP)
    for i in range(P.p):
        lam = float(P.lam[i])
        kkt, g = _restricted_kkt(P.At, P.B[i], lam, X64[i])
        assert kkt <= 1e-6 * lam * 1.01
        off = np.delete(np.abs(g), np.flatnonzero(X64[i]))
        if st["status"][i] == mpl.MPL_SIG_EARLY_STOP:
            assert off.max() <= R * 1.001 + 1e-6 * lam
            assert st["outer_iters"][i] <= rf.stats["outer_iters"][i]
        f = ck.objective(P.At, P.B[i], X64[i], lam)
        f_opt = ck.objective(P.At, P.B[i], X64f[i], lam)
        assert f >= f_opt * (1 - 1e-9)


def test_relative_decrease_rule():
    P = synth.small_problem(256, 1024, 12, 10, 30, rho=4, seed=23, lam_frac=0.01)
    Xf, X64f, rf = solve_gpu(P)
    X, X64, res = solve_gpu(P, stop_eps=1e-2)
    st = res.stats
    assert np.any(st["status"] == mpl.MPL_SIG_EARLY_STOP)
    for i in range(P.p):
        lam = float(P.lam[i])
        kkt, _ = _restricted_kkt(P.At, P.B[i], lam, X64[i])
        assert kkt <= 1e-6 * lam * 1.01
        assert st["outer_iters"][i] <= rf.stats["outer_iters"][i] + 1


@pytest.mark.parametrize("seed", [0, 1])
def test_least_squares_omp(seed):
    """lambda = 0, rho = 1, stop at ||xi|| <= r_2: the atoms of OMP and their
    least-squares fit (Sec. 2.5), against an independent OMP."""
    import torch
    P = synth.small_problem(128, 400, 3, 6, 6, rho=1, seed=500 + seed)
    A = P.At.astype(np.float64)
    r2s, refs = [], []
    for i in range(P.p):
        b = P.B[i].astype(np.float64)
        norms = [np.linalg.norm(b - A.T @ ck.omp(P.At, b, k)[0]) for k in range(1, 12)]
        r2 = 0.5 * (norms[5] + norms[6])  # between the 6th and 7th atom
        r2s.append(r2)
        refs.append(ck.omp(P.At, b, 7))
    for i in range(P.p):
        s = mpl.Solver(torch.from_numpy(P.At).cuda(), rho=1, precision=0, stop_r2=r2s[i], eps_in=1e-7,
                       inner_max=20000)
        X64 = np.zeros((1, P.m))
        Xt = torch.zeros((1, P.m), device="cuda")
        r = s.solve(torch.from_numpy(P.B[i:i + 1]).cuda(), torch.zeros(1, device="cuda"), Xt)
        s.solution_f64(X64)
        s.close()
        assert r.stats["status"][0] == mpl.MPL_SIG_EARLY_STOP
        xo, S = refs[i]
        assert sorted(np.flatnonzero(X64[0]).tolist()) == sorted(S)
        np.testing.assert_allclose(X64[0], xo, rtol=0, atol=1e-6 * np.abs(xo).max())


def _oracle_path(P, i, T):
    """The oracle's exact iterates x^t, t = 0..T (x^0 = 0), of signal i: one solve per prefix
    of the outer loop (max_outer = t), each the exact minimiser on the active set S_t."""
    xs = [np.zeros(P.m)]
    for t in range(1, T + 1):
        x, r, _ = oracle.mpl(P.At, P.B[i], float(P.lam[i]), P.rho, max_outer=t)
        xs.append(x)
    return xs


def _single(P, i):
    return synth.Problem(P.name + f"[{i}]", P.At, P.B[i:i + 1].copy(), P.lam[i:i + 1].copy(), P.rho)


@pytest.mark.parametrize("rule,precision", [("r2", 0), ("r2", 1), ("rinf", 0), ("eps", 0)])
def test_early_stop_parity_midway_thresholds(rule, precision):
    """Each early-stopping rule with its threshold halfway (geometrically) between the values
    the rule sees at two consecutive outer iterations of the oracle's path, so that rounding
    differences between the FP32 iterates and the oracle's exact ones cannot move the
    iteration at which it fires: the GPU must stop at the same active set and return the
    oracle's early-stopped solution (Sec. 2.5, eqs. stop1 and stop_con)."""
    P = synth.small_problem(256, 1024, 4, 24, 36, rho=4, seed=41, lam_frac=0.01)
    A = P.At.astype(np.float64)
    tstar = 3
    for i in range(P.p):
        b = P.B[i].astype(np.float64)
        xs = _oracle_path(P, i, tstar + 1)
        if rule == "r2":
            v = [np.linalg.norm(b - A.T @ x) for x in xs]
            thr = np.sqrt(v[tstar] * v[tstar - 1])
            opts = dict(stop_r2=thr)
        elif rule == "rinf":
            v = [np.abs(A @ (b - A.T @ x)).max() for x in xs]
            thr = np.sqrt(v[tstar] * v[tstar - 1])
            assert thr > P.lam[i] * 1.01
            opts = dict(stop_rinf=thr)
        else:
            lam = float(P.lam[i])
            f = [lam * np.abs(x).sum() + 0.5 * np.sum((b - A.T @ x) ** 2) for x in xs]
            dec = [(f[t - 1] - f[t]) / abs(P.rho * 0.5 * (b @ b)) for t in range(1, tstar + 2)]
            thr = np.sqrt(dec[tstar - 1] * dec[tstar - 2])  # fires after the master problem of t*
            assert dec[tstar - 2] > 1.2 * dec[tstar - 1]
            opts = dict(stop_eps=thr)
        # the oracle with the rule on
        key = {"stop_r2": "stop_r2", "stop_rinf": "stop_rinf", "stop_eps": "stop_eps"}
        xo, ro, _ = oracle.mpl(P.At, P.B[i], float(P.lam[i]), P.rho, **{key[k]: v for k, v in opts.items()})
        assert ro["status"] == 3, (rule, i, ro)
        Pi = _single(P, i)
        X, X64, res = solve_gpu(Pi, precision=precision, **opts)
        st = res.stats
        assert st["status"][0] == mpl.MPL_SIG_EARLY_STOP, (rule, i, st["status"])
        assert st["active_size"][0] == ro["S_size"], (rule, i, st["active_size"][0], ro["S_size"])
        check_against_oracle(Pi, X64, xo[None, :], [0])
