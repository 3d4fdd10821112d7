"""The identity route of the worst-case analysis (Sec. 3, eq. "batchQ"):
g = beta - Q_S x_S with Q = A^T A and beta = A^T b, and the autotuner that
decides when to take it.

The selection widens its re-score band to the route's rigorous error bound and
ranks by the same fixed-order FP32 re-score as the GEMM route, so a solve that
takes the identity route at some or all iterations must pick the same atoms at
every outer iteration and return bit-identical solutions.  The oracle's own
identity route (corr_route = 1) is pinned against its direct route on CPU; here
the GPU route is checked against the GPU GEMM route and the FP64 oracle.

The Gram growth read out of Q (MPL_OPT_QGRAM) gives the same G and h bits as
the computed Gram block (one FMA chain per entry, k ascending, on both
sides), so every solve with it must equal the one without it bit for bit."""
import numpy as np
import pytest

from paper_1302_5010_gb300 import mpl, synth
from parity import check_against_oracle
from test_gpu_parity import assert_certified, oracle_solve, solve_gpu

pytestmark = pytest.mark.gpu


def _qcols(P, precision, qroute, **opts):
    import torch
    s = mpl.Solver(torch.from_numpy(P.At).cuda(), rho=P.rho, precision=precision, qroute=qroute, **opts)
    X = torch.empty((P.p, P.m), dtype=torch.float32, device="cuda")
    s.solve(torch.from_numpy(P.B).cuda(), torch.from_numpy(P.lam).cuda(), X)
    torch.cuda.synchronize()
    ph = s.phase_times()
    s.close()
    return ph["qroute_columns"], ph["corr_columns"]


@pytest.mark.parametrize("precision", [0, 1])
def test_identity_route_matches_gemm_route_c2(precision):
    P = synth.make_config("c2", p=64)
    Xg, X64g, rg = solve_gpu(P, precision=precision, reentry=1)
    Xq, X64q, rq = solve_gpu(P, precision=precision, qroute=1024, reentry=1)
    assert_certified(rg)
    assert_certified(rq)
    np.testing.assert_array_equal(rg.stats["outer_iters"], rq.stats["outer_iters"])
    np.testing.assert_array_equal(rg.stats["active_size"], rq.stats["active_size"])
    np.testing.assert_array_equal(Xg, Xq)
    np.testing.assert_array_equal(X64g, X64q)
    qc, cc = _qcols(P, precision, 1024)
    assert qc > 0 and qc < cc  # every iteration after the first read Q


def test_identity_route_first_iterations_only():
    P = synth.make_config("c2", p=48)
    Xg, _, rg = solve_gpu(P, precision=1, reentry=1)
    Xq, _, rq = solve_gpu(P, precision=1, qroute=2 * P.rho, reentry=1)  # iterations 1 and 2 only
    assert_certified(rq)
    np.testing.assert_array_equal(Xg, Xq)
    qc, cc = _qcols(P, 1, 2 * P.rho)
    assert 0 < qc <= 2 * P.p


@pytest.mark.parametrize("n,m,p,rho", [(256, 1000, 19, 5), (198, 777, 9, 3)])
def test_identity_route_ragged_against_oracle(n, m, p, rho):
    """m % 4 != 0 takes the scalar path of the route; n % 4 != 0 the scalar GEMM."""
    P = synth.small_problem(n, m, p, 4, min(30, n // 6), rho=rho, seed=n + 7 * m + p, lam_frac=0.03)
    X, X64, res = solve_gpu(P, precision=0, qroute=1024, reentry=1)
    assert_certified(res)
    check_against_oracle(P, X64, oracle_solve(P))
    Xg, _, _ = solve_gpu(P, precision=0, reentry=1)
    np.testing.assert_array_equal(X, Xg)


def test_identity_route_warm_start():
    """The route's bound on |S| counts the atoms a warm start admits."""
    import torch
    P = synth.make_config("c2", p=32)
    Pt = synth.make_config("c2", p=1024, seed_shift=9000)
    s = mpl.Solver(torch.from_numpy(P.At).cuda(), rho=P.rho, precision=1, reentry=1)
    Xt = torch.empty((Pt.p, Pt.m), device="cuda")
    s.solve(torch.from_numpy(Pt.B).cuda(), torch.from_numpy(Pt.lam).cuda(), Xt)
    s.train_proposal(torch.from_numpy(Pt.B).cuda(), torch.from_numpy(Pt.lam).cuda(), Xt, epochs=2)
    s.set(mpl.MPL_OPT_WARM_START, 2)
    B, lam = torch.from_numpy(P.B).cuda(), torch.from_numpy(P.lam).cuda()
    X0 = torch.empty((P.p, P.m), device="cuda")
    r0 = s.solve(B, lam, X0)
    s.set(mpl.MPL_OPT_QROUTE, 1024)
    X1 = torch.empty((P.p, P.m), device="cuda")
    r1 = s.solve(B, lam, X1)
    torch.cuda.synchronize()
    assert np.all(r0.stats["status"] == mpl.MPL_SIG_CERTIFIED)
    assert np.all(r1.stats["status"] == mpl.MPL_SIG_CERTIFIED)
    assert torch.equal(X0, X1)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_gram_from_q_is_bit_identical_c2(precision):
    P = synth.make_config("c2", p=64)
    Xg, X64g, rg = solve_gpu(P, precision=precision, reentry=1)
    Xq, X64q, rq = solve_gpu(P, precision=precision, qgram=1, reentry=1)
    assert_certified(rq)
    for k in ("outer_iters", "inner_iters", "active_size", "finishes"):
        np.testing.assert_array_equal(rg.stats[k], rq.stats[k])
    np.testing.assert_array_equal(Xg, Xq)
    np.testing.assert_array_equal(X64g, X64q)


@pytest.mark.parametrize("n,m,p,rho,omega", [(198, 777, 9, 3, 1), (260, 1000, 13, 5, 1), (256, 1000, 11, 4, 3)])
def test_gram_from_q_ragged(n, m, p, rho, omega):
    """n % 4 != 0: the scalar Gram kernel and the selection's scalar re-score (which forms h);
    n % 16 != 0: ragged K slices; omega > 1: Algorithm 2's explored atoms."""
    P = synth.small_problem(n, m, p, 4, min(30, n // 6), rho=rho, seed=3 * n + m + p, lam_frac=0.03)
    Xg, _, _ = solve_gpu(P, precision=0, omega=omega, reentry=1)
    X, X64, res = solve_gpu(P, precision=0, omega=omega, qgram=1, reentry=1)
    assert_certified(res)
    np.testing.assert_array_equal(X, Xg)
    check_against_oracle(P, X64, oracle_solve(P))


def test_gram_from_q_with_identity_route_and_warm_start():
    import torch
    P = synth.make_config("c2", p=32)
    Pt = synth.make_config("c2", p=1024, seed_shift=9000)
    s = mpl.Solver(torch.from_numpy(P.At).cuda(), rho=P.rho, precision=1, reentry=1)
    Xt = torch.empty((Pt.p, Pt.m), device="cuda")
    s.solve(torch.from_numpy(Pt.B).cuda(), torch.from_numpy(Pt.lam).cuda(), Xt)
    s.train_proposal(torch.from_numpy(Pt.B).cuda(), torch.from_numpy(Pt.lam).cuda(), Xt, epochs=2)
    s.set(mpl.MPL_OPT_WARM_START, 2)
    B, lam = torch.from_numpy(P.B).cuda(), torch.from_numpy(P.lam).cuda()
    X0 = torch.empty((P.p, P.m), device="cuda")
    s.solve(B, lam, X0)
    s.set(mpl.MPL_OPT_QGRAM, 1)
    s.set(mpl.MPL_OPT_QROUTE, 2 * P.rho)
    X1 = torch.empty((P.p, P.m), device="cuda")
    r1 = s.solve(B, lam, X1)
    torch.cuda.synchronize()
    assert np.all(r1.stats["status"] == mpl.MPL_SIG_CERTIFIED)
    assert torch.equal(X0, X1)
    s.close()


def test_autotune_keeps_the_solution():
    import torch
    P = synth.make_config("c2", p=64)
    s = mpl.Solver(torch.from_numpy(P.At).cuda(), rho=P.rho, precision=1, reentry=1)
    B, lam = torch.from_numpy(P.B).cuda(), torch.from_numpy(P.lam).cuda()
    X0 = torch.empty((P.p, P.m), device="cuda")
    s.solve(B, lam, X0)
    t = s.autotune(B, lam)
    assert t["candidates"] >= 3
    assert t["sync_every"] in (1, 2, 4)
    assert t["qroute"] in [0] + [min(256, k * P.rho) for k in (1, 2, 4)]
    assert t["qgram"] in (0, 1) and t["candidates"] >= 12  # Q fits: both stages ran
    assert 0 < t["ms"] <= t["ms_default"] + 1e-9
    assert s.h is not None and mpl.mpl_get_option(s.h, mpl.MPL_OPT_QROUTE) == t["qroute"]
    assert mpl.mpl_get_option(s.h, mpl.MPL_OPT_SYNC_EVERY) == t["sync_every"]
    assert mpl.mpl_get_option(s.h, mpl.MPL_OPT_QGRAM) == t["qgram"]
    X1 = torch.empty((P.p, P.m), device="cuda")
    r = s.solve(B, lam, X1)
    torch.cuda.synchronize()
    assert np.all(r.stats["status"] == mpl.MPL_SIG_CERTIFIED)
    assert torch.equal(X0, X1)
    s.close()
