"""Failure detection on the host side (no device fault is provoked).

- A signal whose column of B holds a NaN is reported MPL_SIG_NONFINITE; the
  other signals of the same batch are certified and their solutions are the
  ones a batch without the poisoned column gives (signals are independent,
  eq. 3).
- MPL_OPT_MAX_OUTER = 1 stops every signal after one worst-case analysis: the
  status is MPL_SIG_MAX_OUTER, the call returns MPL_ERR_NOT_CONVERGED, and the
  returned x is the exact minimiser of eq. 2 restricted to the rho atoms the
  analysis added, the oracle's answer with one outer iteration."""
import numpy as np
import pytest

import oracle
from paper_1302_5010_gb300 import mpl, synth
from parity import check_against_oracle
from test_gpu_parity import TOL, assert_certified, solve_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_column_isolated(precision):
    P = synth.make_config("c2", p=24)
    bad = 5
    B = P.B.copy()
    B[bad, 17] = np.nan
    Q = synth.Problem("nan", P.At, B, P.lam.copy(), P.rho)
    X, X64, res = solve_gpu(Q, precision=precision, reentry=1)
    st = res.stats
    assert res.status == mpl.MPL_ERR_NOT_CONVERGED
    assert st["status"][bad] == mpl.MPL_SIG_NONFINITE
    others = np.array([i for i in range(P.p) if i != bad])
    assert np.all(st["status"][others] == mpl.MPL_SIG_CERTIFIED), st["status"]
    assert np.all(st["kkt"][others] <= TOL)
    assert np.all(X[bad] == 0)
    # the clean batch without the poisoned column gives the same solutions, bit for bit
    Pc = P.subset(others)
    Xc, _, rc = solve_gpu(Pc, precision=precision, reentry=1)
    assert_certified(rc)
    np.testing.assert_array_equal(X[others], Xc)


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_column_isolated_long_score_rows(precision):
    """Score rows above the shared-memory row cache (2048 x 32768): the chunk maxima flag the
    poisoned signal's non-finite scores; the flag stays with that signal, whose selection
    stops at once, and does not reach the signal that takes its place in the next
    iteration's active list."""
    P = synth.make_config("c5", p=24)
    bad = 3
    B = P.B.copy()
    B[bad, 11] = np.nan
    Q = synth.Problem("nan-c5", P.At, B, P.lam.copy(), P.rho)
    X, X64, res = solve_gpu(Q, precision=precision, smax=512, reentry=1)
    st = res.stats
    assert res.status == mpl.MPL_ERR_NOT_CONVERGED
    assert st["status"][bad] == mpl.MPL_SIG_NONFINITE
    others = np.array([i for i in range(P.p) if i != bad])
    assert np.all(st["status"][others] == mpl.MPL_SIG_CERTIFIED), st["status"]
    assert np.all(X[bad] == 0)
    Xc, _, rc = solve_gpu(P.subset(others), precision=precision, smax=512, reentry=1)
    assert_certified(rc)
    np.testing.assert_array_equal(X[others], Xc)


def test_nan_lambda_and_inf_signal():
    P = synth.small_problem(256, 1024, 6, 5, 12, rho=4, seed=31, lam_frac=0.03)
    B = P.B.copy()
    B[1, 0] = np.inf
    lam = P.lam.copy()
    lam[4] = np.nan
    Q = synth.Problem("nonfinite", P.At, B, lam, P.rho)
    X, X64, res = solve_gpu(Q)
    st = res.stats
    assert st["status"][1] == mpl.MPL_SIG_NONFINITE and st["status"][4] == mpl.MPL_SIG_NONFINITE
    ok = [0, 2, 3, 5]
    assert np.all(st["status"][ok] == mpl.MPL_SIG_CERTIFIED)
    Xo, r = oracle.bmpl(P.At, P.B[ok], P.lam[ok], P.rho)
    check_against_oracle(P, X64[ok], Xo, ok)


def test_max_outer_one():
    P = synth.make_config("c2", p=16)
    X, X64, res = solve_gpu(P, max_outer=1)
    st = res.stats
    assert res.status == mpl.MPL_ERR_NOT_CONVERGED
    # every c2 signal has more than rho = 15 violators at x = 0 (k >= 20)
    assert np.all(st["status"] == mpl.MPL_SIG_MAX_OUTER), st["status"]
    assert np.all(st["active_size"] == P.rho)
    assert np.all(st["outer_iters"] >= 1)
    A64 = P.At.astype(np.float64)
    for i in range(P.p):
        b = P.B[i].astype(np.float64)
        f = float(P.lam[i]) * np.abs(X64[i]).sum() + 0.5 * np.sum((b - A64.T @ X64[i]) ** 2)
        assert f < 0.5 * b @ b  # strictly below f(0): the rho atoms were used
    # the oracle stopped after one outer iteration solves the same restricted problem
    Xo, r = oracle.bmpl(P.At, P.B, P.lam, P.rho, max_outer=1)
    assert np.all(r["status"] == 1) and np.all(r["S_size"] == P.rho)
    check_against_oracle(P, X64, Xo)
