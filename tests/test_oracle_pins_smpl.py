"""Pins for the oracle's subspace exploratory matching (SMPL, Algorithm 2) and
its early-stopping rules (Sec. 2.5, eqs. stop1 and stop_con), each reached by
something other than the oracle itself.

  other solver   SMPL still ends at the LASSO minimiser: coordinate descent
                 and brute-force sign enumeration agree with it
  brute force    the atom SMPL keeps at the first iteration is the one with
                 the largest |u| of the LASSO restricted to the omega*rho
                 largest correlations, solved by sign enumeration; on the
                 constructed dictionary it differs from MPL's first atom
  sort           the kept atoms are among the omega*rho largest |a_j^T b|
  reduction      lambda = 0, rho = 1 with the residual rule ||xi|| <= r_2
                 stops where an independent OMP first reaches r_2
  placement      a stop by ||A^T xi||_inf <= r_inf or by the relative decrease
                 returns the iterate that a run capped at the same number of
                 master problems returns, and the rule did not hold one step
                 earlier (objectives and correlations recomputed in numpy)
"""
import numpy as np
import pytest

import oracle
from oracle import checkers as ck
from paper_1302_5010_gb300 import synth


def _unit_rows(M):
    return M / np.linalg.norm(M, axis=1, keepdims=True)


@pytest.mark.parametrize("omega", [2, 3, 5])
@pytest.mark.parametrize("seed", [0, 1])
def test_smpl_reaches_the_lasso_minimiser(omega, seed):
    P = synth.small_problem(64, 160, 1, 8, 12, rho=3, seed=300 + seed, lam_frac=0.05)
    b = P.B[0].astype(np.float64)
    lam = float(P.lam[0])
    x, res, tr = oracle.mpl(P.At, b, lam, P.rho, omega=omega)
    assert res["status"] == 0
    xc = ck.cd_lasso(P.At, b, lam)
    np.testing.assert_allclose(x, xc, rtol=0, atol=1e-8)
    assert ck.kkt_violation(P.At, b, x, lam) < 1e-9


@pytest.mark.parametrize("omega", [2, 4])
def test_smpl_bruteforce_tiny(omega):
    rng = np.random.default_rng(5)
    At = _unit_rows(rng.standard_normal((9, 6)))
    b = rng.standard_normal(6)
    lam = 0.1 * np.max(np.abs(At @ b))
    x, res, _ = oracle.mpl(At, b, lam, 1, omega=omega)
    xb = ck.bruteforce_lasso(At, b, lam)
    np.testing.assert_allclose(x, xb, rtol=0, atol=1e-9)


def _wedge():
    """a1 = e1, a3 = e2, and a2 between them with a component off their plane:
    b = a1 + 0.9 a3 correlates most with a2, which cannot represent b."""
    a1 = np.array([1.0, 0.0, 0.0])
    a3 = np.array([0.0, 1.0, 0.0])
    a2 = np.array([1.0, 1.0, 0.5])
    a2 /= np.linalg.norm(a2)
    a4 = np.array([0.3, -0.2, 1.0])
    a4 /= np.linalg.norm(a4)
    At = np.stack([a1, a2, a3, a4])
    b = a1 + 0.9 * a3
    return At, b


def test_smpl_keeps_largest_restricted_coefficient():
    At, b = _wedge()
    lam = 0.05
    g = At @ b
    order = sorted(range(4), key=lambda j: (-abs(g[j]), j))
    assert order[0] == 1  # the largest correlation is a2
    # MPL (rho = 1) takes a2 first
    _, _, tr1 = oracle.mpl(At, b, lam, 1)
    assert int(tr1["added"][0][0]) == 1
    # SMPL with omega = 3: LASSO on the three largest, by sign enumeration
    J = order[:3]
    u = ck.bruteforce_lasso(At[J], b, lam)
    keep = J[int(np.argmax(np.abs(u)))]
    assert keep != 1
    x, res, tr3 = oracle.mpl(At, b, lam, 1, omega=3)
    assert int(tr3["added"][0][0]) == keep
    # and both still end at the LASSO minimiser
    xb = ck.bruteforce_lasso(At, b, lam)
    np.testing.assert_allclose(x, xb, rtol=0, atol=1e-9)


def test_smpl_first_atoms_among_top_correlations():
    P = synth.small_problem(128, 512, 1, 10, 20, rho=4, seed=77, lam_frac=0.03)
    b = P.B[0].astype(np.float64)
    omega = 3
    _, _, tr = oracle.mpl(P.At, b, float(P.lam[0]), P.rho, omega=omega)
    g = np.abs(P.At.astype(np.float64) @ b)
    top = set(np.argsort(-g, kind="stable")[: omega * P.rho].tolist())
    first = [int(j) for j in tr["added"][0]]
    assert len(first) == P.rho
    assert set(first) <= top


@pytest.mark.parametrize("seed", [0, 1])
def test_omp_residual_rule(seed):
    P = synth.small_problem(64, 200, 1, 6, 6, rho=1, seed=90 + seed)
    b = P.B[0].astype(np.float64)
    # the independent OMP's residual norms, step by step
    norms = []
    for k in range(1, 16):
        xo, S = ck.omp(P.At, b, k)
        norms.append(np.linalg.norm(b - P.At.astype(np.float64).T @ xo))
    r2 = 0.5 * (norms[6] + norms[7])  # between steps 7 and 8
    kstop = next(k for k, v in enumerate(norms, start=1) if v <= r2)
    x, res, tr = oracle.mpl(P.At, b, 0.0, 1, stop_r2=r2)
    assert res["status"] == 3
    xo, S = ck.omp(P.At, b, kstop)
    assert [int(a[0]) for a in tr["added"] if len(a)] == S
    np.testing.assert_allclose(x, xo, rtol=0, atol=1e-9)


def _run(P, b, lam, **kw):
    return oracle.mpl(P.At, b, lam, P.rho, **kw)


def test_rinf_rule_placement():
    P = synth.small_problem(96, 300, 1, 10, 14, rho=2, seed=41, lam_frac=0.02)
    b = P.B[0].astype(np.float64)
    lam = float(P.lam[0])
    A = P.At.astype(np.float64)
    ginf = lambda x: np.max(np.abs(A @ (b - A.T @ x)))
    x_full, r_full, _ = _run(P, b, lam)
    T = r_full["n_outer"]
    # a threshold the iterates cross half way
    x_mid, _, _ = _run(P, b, lam, max_outer=T // 2)
    rinf = 1.01 * ginf(x_mid)
    x, res, tr = _run(P, b, lam, stop_rinf=rinf)
    assert res["status"] == 3
    k = res["n_outer"] - 1  # master problems solved before the stop
    xk, _, _ = _run(P, b, lam, max_outer=k)
    np.testing.assert_array_equal(x, xk)
    assert ginf(x) <= rinf
    if k > 0:
        xk1, _, _ = _run(P, b, lam, max_outer=k - 1) if k > 1 else (np.zeros_like(x), None, None)
        assert ginf(xk1) > rinf


def test_relative_decrease_rule_placement():
    P = synth.small_problem(96, 300, 1, 10, 14, rho=2, seed=43, lam_frac=0.02)
    b = P.B[0].astype(np.float64)
    lam = float(P.lam[0])
    f0 = 0.5 * float(b @ b)
    f = lambda x: ck.objective(P.At, b, x, lam)
    fs = [f0]
    for k in range(1, 9):
        xk, _, _ = _run(P, b, lam, max_outer=k)
        fs.append(f(xk))
    dec = [(fs[t - 1] - fs[t]) / abs(P.rho * f0) for t in range(1, len(fs))]
    eps = 0.5 * (dec[3] + dec[4]) if dec[3] > dec[4] else 0.99 * dec[4]
    tstop = next(t for t, v in enumerate(dec, start=1) if v <= eps)
    x, res, _ = _run(P, b, lam, stop_eps=eps)
    assert res["status"] == 3
    xk, _, _ = _run(P, b, lam, max_outer=tstop)
    np.testing.assert_array_equal(x, xk)
    assert abs(res["objective"] - f(x)) <= 1e-12 * f0
