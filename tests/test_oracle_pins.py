"""Pins for the FP64 MPL oracle: facts fixed by the paper and by the mathematics
of eq. 2, each reached by something other than the oracle itself.

  closed form    orthonormal A: x = soft(A^T b, lambda)
  special case   lambda >= ||A^T b||_inf  =>  x = 0 and J_1 is empty (Sec. 2.3)
  brute force    sign enumeration on tiny problems (n < m and n >= m), and a
                 stored fixture written by tests/golden/make_golden.py
  other solver   cyclic coordinate descent
  optimality     KKT of eq. 2 and the duality gap with the dual point of eq. 5,
                 evaluated in numpy
  reduction      lambda = 0, rho = 1  =>  OMP, iteration by iteration (Sec. 2.3)
  invariants     monotone f over outer iterations (no deletion, Sec. 2.2);
                 Lemma 1's decrease bound for the first PG step
  selection      top-rho by |g_j|, ties to the lower index, against a sort
  batch mode     the BMPL identity route (eq. batchQ) equals the direct route
"""
import os

import numpy as np
import pytest

import oracle
from oracle import checkers as ck
from paper_1302_5010_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tiny_lasso.txt")


def _unit_rows(M):
    return M / np.linalg.norm(M, axis=1, keepdims=True)


@pytest.mark.parametrize("rho", [1, 3, 8])
@pytest.mark.parametrize("frac", [0.05, 0.3, 0.9])
def test_orthonormal_closed_form(rho, frac):
    rng = np.random.default_rng(11 + rho)
    Q, _ = np.linalg.qr(rng.standard_normal((48, 48)))
    At = Q.T.copy()
    b = rng.standard_normal(48)
    lam = frac * np.abs(At @ b).max()
    x, res, _ = oracle.mpl(At, b, lam, rho)
    ref = ck.soft_threshold_orthonormal(At, b, lam)
    assert res["status"] == 0
    np.testing.assert_allclose(x, ref, rtol=0, atol=1e-12)


def test_lambda_above_max_gives_zero():
    P = synth.small_problem(64, 256, 1, 5, 5, rho=4, seed=3)
    b = P.B[0].astype(np.float64)
    lam = np.abs(P.At.astype(np.float64) @ b).max() * (1 + 1e-12)
    x, res, tr = oracle.mpl(P.At, b, lam, 4)
    assert np.all(x == 0)
    assert res["n_outer"] == 1 and tr["n_added"][0] == 0 and res["status"] == 0


@pytest.mark.parametrize("seed,n,m", [(0, 5, 7), (1, 6, 8), (2, 8, 6), (3, 4, 8), (4, 7, 7)])
def test_bruteforce_tiny(seed, n, m):
    rng = np.random.default_rng(100 + seed)
    At = _unit_rows(rng.standard_normal((m, n)))
    b = rng.standard_normal(n)
    for frac in (0.02, 0.2, 0.6):
        lam = frac * np.abs(At @ b).max()
        xb = ck.bruteforce_lasso(At, b, lam)
        for rho in (1, 2, 3):
            x, res, _ = oracle.mpl(At, b, lam, rho)
            np.testing.assert_allclose(x, xb, rtol=0, atol=1e-10)


def test_golden_fixture():
    with open(GOLDEN) as f:
        rows = [ln.split() for ln in f if not ln.startswith("#")]
    n, m = int(rows[0][0]), int(rows[0][1])
    lam = float(rows[1][0])
    b = np.array(rows[2], dtype=np.float64)
    At = np.array(rows[3:3 + m], dtype=np.float64)
    xs = np.array(rows[3 + m], dtype=np.float64)
    assert At.shape == (m, n)
    for rho in (1, 2, 4):
        x, res, _ = oracle.mpl(At, b, lam, rho)
        np.testing.assert_allclose(x, xs, rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1])
def test_coordinate_descent_agrees(seed):
    P = synth.small_problem(128, 512, 1, 8, 20, rho=4, seed=40 + seed, lam_frac=0.03)
    b = P.B[0].astype(np.float64)
    lam = float(P.lam[0])
    x, res, _ = oracle.mpl(P.At, b, lam, P.rho)
    xc = ck.cd_lasso(P.At, b, lam)
    assert res["status"] == 0
    np.testing.assert_allclose(x, xc, rtol=0, atol=1e-9 * max(1.0, np.abs(xc).max()))


def test_c1_workload_optimal():
    P = synth.make_config("c1")
    b = P.B[0].astype(np.float64)
    lam = float(P.lam[0])
    x, res, tr = oracle.mpl(P.At, b, lam, P.rho)
    assert res["status"] == 0
    assert ck.kkt_violation(P.At, b, x, lam) < 1e-10
    assert ck.duality_gap(P.At, b, x, lam) < 1e-12
    xc = ck.cd_lasso(P.At, b, lam)
    np.testing.assert_allclose(x, xc, rtol=0, atol=1e-9)
    # the oracle's own certificate agrees with the numpy one
    assert abs(res["kkt"] - ck.kkt_violation(P.At, b, x, lam)) < 1e-12


def test_batch_kkt_and_gap():
    P = synth.small_problem(256, 2048, 6, 10, 30, rho=8, seed=5)
    X, res = oracle.bmpl(P.At, P.B, P.lam, P.rho, threads=2)
    for i in range(P.p):
        b = P.B[i].astype(np.float64)
        assert ck.kkt_violation(P.At, b, X[i], float(P.lam[i])) < 1e-9
        assert ck.duality_gap(P.At, b, X[i], float(P.lam[i])) < 1e-11
    assert np.all(res["status"] == 0)


def test_batch_equals_single():
    P = synth.small_problem(96, 384, 4, 4, 12, rho=3, seed=9)
    X, res = oracle.bmpl(P.At, P.B, P.lam, P.rho, threads=3)
    for i in range(P.p):
        x, r, _ = oracle.mpl(P.At, P.B[i], P.lam[i], P.rho)
        np.testing.assert_array_equal(x, X[i])
        assert r["n_outer"] == res["n_outer"][i]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_omp_reduction(seed):
    """lambda = 0, rho = 1: MPL picks the OMP atoms in the same order and x is
    the least-squares fit on them (Sec. 2.3)."""
    P = synth.small_problem(64, 200, 1, 6, 6, rho=1, seed=60 + seed)
    b = P.B[0].astype(np.float64)
    k = 9
    x, res, tr = oracle.mpl(P.At, b, 0.0, 1, max_outer=k)
    xo, S = ck.omp(P.At, b, k)
    picked = [int(a[0]) for a in tr["added"]]
    assert picked == S
    np.testing.assert_allclose(x, xo, rtol=0, atol=1e-9)


@pytest.mark.parametrize("rho", [1, 4, 16])
def test_monotone_objective_and_lemma1(rho):
    """f(x^t) never increases (atoms are never deleted), and the first PG
    step of outer iteration t decreases f by at least
    (1/2L) * sum_{i in J_t} (|g_i| - lambda)^2 (Lemma 1)."""
    P = synth.small_problem(256, 1024, 1, 25, 25, rho=rho, seed=70 + rho, lam_frac=0.01)
    b = P.B[0].astype(np.float64)
    lam = float(P.lam[0])
    x, res, tr = oracle.mpl(P.At, b, lam, rho)
    T = res["n_outer"]
    f = tr["f_iter"][: T - 1]
    assert np.all(np.diff(f) <= 1e-12 * f[0])
    assert np.all(tr["f_prev"][1:T - 1] == f[:-1])
    for t in range(T - 1):
        g = np.asarray(tr["gsel"][t])
        bound = ((g - lam) ** 2).sum() / (2.0 * tr["L_first"][t])
        dec = tr["f_prev"][t] - tr["f_first"][t]
        assert dec >= bound * (1 - 1e-9) - 1e-13, (t, dec, bound)


def test_selection_order_with_ties():
    """With A = I, g = b at t = 1: the ranked violators are |b_j| > lambda,
    larger first and the lower index first among equal magnitudes."""
    b = np.array([0.5, -0.9, 0.9, 0.1, 0.9, -0.5, 0.3, 0.05])
    At = np.eye(8)
    lam = 0.2
    x, res, tr = oracle.mpl(At, b, lam, 4)
    assert list(tr["added"][0]) == [1, 2, 4, 0]
    assert list(tr["added"][1]) == [5, 6]
    assert tr["n_added"][2] == 0
    order = sorted(range(8), key=lambda j: (-abs(b[j]), j))
    assert [j for j in order if abs(b[j]) > lam] == [1, 2, 4, 0, 5, 6]
    np.testing.assert_allclose(x, np.sign(b) * np.maximum(np.abs(b) - lam, 0), atol=1e-14)


def test_batch_identity_route():
    """The worst-case analysis through beta - Q_I x_I (eq. batchQ) selects the
    same atoms and reaches the same solution as A^T xi."""
    P = synth.small_problem(80, 300, 3, 5, 15, rho=4, seed=21)
    for i in range(P.p):
        b = P.B[i].astype(np.float64)
        x0, r0, t0 = oracle.mpl(P.At, b, P.lam[i], 4, corr_route=0)
        x1, r1, t1 = oracle.mpl(P.At, b, P.lam[i], 4, corr_route=1)
        assert [list(a) for a in t0["added"]] == [list(a) for a in t1["added"]]
        np.testing.assert_allclose(x1, x0, rtol=0, atol=1e-11)
    X0, _ = oracle.bmpl(P.At, P.B, P.lam, 4, corr_route=0)
    X1, _ = oracle.bmpl(P.At, P.B, P.lam, 4, corr_route=1)
    np.testing.assert_allclose(X1, X0, rtol=0, atol=1e-11)


def test_edge_cases():
    P = synth.small_problem(32, 64, 2, 3, 3, rho=2, seed=1)
    X, res = oracle.bmpl(P.At, P.B[:0], P.lam[:0], 2)
    assert X.shape == (0, 64)
    x, r, _ = oracle.mpl(P.At, np.zeros(32), 0.1, 2)
    assert np.all(x == 0) and r["n_outer"] == 1
    # rho larger than the number of violators: takes all of them at once
    x, r, tr = oracle.mpl(P.At, P.B[0], P.lam[0], 64)
    assert r["status"] == 0 and ck.kkt_violation(P.At, P.B[0], x, float(P.lam[0])) < 1e-10


@pytest.mark.parametrize("frac", [0.1, 0.4, 0.8])
def test_gap_closed_form_orthonormal_at_zero(frac):
    """Dual of eq. 5 with the scaled dual point alpha = r min(1, lambda/||A^T r||_inf): for an
    orthonormal A at x = 0 (r = b, P = ||b||^2 / 2) the point is alpha = c b with
    c = lambda/||A^T b||_inf, D = c ||b||^2 - c^2 ||b||^2 / 2, and the relative gap is
    (P - D)/P = (1 - c)^2 (worked out by hand).  A sign slip in D, a wrong dual scale or a
    division by D instead of P moves the value off this curve."""
    rng = np.random.default_rng(70 + int(frac * 10))
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    At = Q.T.copy()
    b = rng.standard_normal(40)
    lam = frac * np.abs(At @ b).max()
    c = oracle.certify(At, b, lam, np.zeros(40))
    assert c["gap"] == pytest.approx((1.0 - frac) ** 2, rel=1e-12)
    assert c["objective"] == pytest.approx(0.5 * b @ b, rel=1e-14)


def test_gap_weak_duality_and_checker_agreement():
    """At points away from the optimum the oracle's gap bounds the true suboptimality from
    above (weak duality: D(alpha) <= P*, with P* from the independent coordinate-descent
    solver), vanishes at the optimum, and agrees with the numpy certificate."""
    P = synth.small_problem(96, 300, 3, 4, 10, rho=3, seed=71, lam_frac=0.05)
    rng = np.random.default_rng(5)
    for i in range(P.p):
        b = P.B[i].astype(np.float64)
        lam = float(P.lam[i])
        xs = ck.cd_lasso(P.At, b, lam)
        fstar = ck.objective(P.At, b, xs, lam)
        c_opt = oracle.certify(P.At, b, lam, xs)
        assert abs(c_opt["gap"]) < 1e-10
        for scale in (0.0, 0.5, 0.9, 1.2):
            x = scale * xs + (0.0 if scale == 0 else 0.01) * rng.standard_normal(P.m) * (xs != 0)
            c = oracle.certify(P.At, b, lam, x)
            f = ck.objective(P.At, b, x, lam)
            assert c["objective"] == pytest.approx(f, rel=1e-12)
            assert c["gap"] >= (f - fstar) / f - 1e-12
            assert c["gap"] == pytest.approx(ck.duality_gap(P.At, b, x, lam), rel=1e-9, abs=1e-14)
