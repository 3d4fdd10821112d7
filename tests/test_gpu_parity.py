"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Small cases compare every signal; the full 1024 x 8192, p = 256 workload (the
benchmark's configuration) compares a sample of signals one by one and checks
the certificate of every signal in FP64."""
import numpy as np
import pytest

import oracle
from oracle import checkers as ck
from paper_1302_5010_gb300 import mpl, synth
from parity import check_against_oracle

pytestmark = pytest.mark.gpu
TOL = 1e-6


def _torch():
    import torch
    return torch


def solve_gpu(P, precision=0, tol=TOL, host=False, **opts):
    torch = _torch()
    solver = mpl.Solver(torch.from_numpy(P.At).cuda() if not host else P.At, rho=P.rho,
                        precision=precision, **opts)
    if host:
        X = np.zeros((P.p, P.m), dtype=np.float32)
        res = solver.solve(P.B, P.lam, X, tol)
    else:
        B = torch.from_numpy(P.B).cuda()
        lam = torch.from_numpy(P.lam).cuda()
        Xt = torch.empty((P.p, P.m), dtype=torch.float32, device="cuda")
        res = solver.solve(B, lam, Xt, tol)
        torch.cuda.synchronize()
        X = Xt.cpu().numpy()
    X64 = np.zeros((P.p, P.m), dtype=np.float64)
    solver.solution_f64(X64)
    solver.close()
    return X, X64, res


def oracle_solve(P, idx=None):
    idx = np.arange(P.p) if idx is None else np.asarray(idx)
    X, r = oracle.bmpl(P.At, P.B[idx], P.lam[idx], P.rho)
    assert np.all(r["status"] == 0)
    return X


def assert_certified(res):
    st = res.stats
    assert np.all(st["status"] == mpl.MPL_SIG_CERTIFIED), st["status"]
    assert np.all(st["kkt"] <= TOL), st["kkt"].max()
    assert res.status == mpl.MPL_OK


def test_c1_single_signal():
    P = synth.make_config("c1")
    X, X64, res = solve_gpu(P)
    assert_certified(res)
    Xo = oracle_solve(P)
    check_against_oracle(P, X, Xo)
    check_against_oracle(P, X64, Xo)
    # the GPU's certificate is an upper bound: the FP64 recomputation stays below it
    kkt64 = ck.kkt_violation(P.At, P.B[0], X64[0], float(P.lam[0]))
    assert kkt64 <= TOL * (1 + 1e-9)
    assert kkt64 <= res.stats["kkt"][0] * (1 + 1e-9) + 1e-12


@pytest.mark.parametrize("n,m,p,rho", [(256, 1000, 37, 5), (250, 777, 9, 3), (512, 4096, 130, 12)])
def test_ragged_shapes(n, m, p, rho):
    """Several GEMM tiles with ragged tails in atoms, signals and (n % 4 != 0) length."""
    P = synth.small_problem(n, m, p, 5, min(40, n // 6), rho=rho, seed=n + m + p, lam_frac=0.03)
    X, X64, res = solve_gpu(P)
    assert_certified(res)
    check_against_oracle(P, X64, oracle_solve(P))


def test_long_signals_residual_in_global_memory():
    """n > 4096: the exact finish keeps its double-FP32 residual in the signal's global rows
    instead of shared memory (the layout it also takes when more signals finish at once than
    there are SMs and the shared-memory one fits a single CTA per SM)."""
    P = synth.small_problem(4104, 3000, 12, 20, 60, rho=10, seed=4104, lam_frac=0.02)
    for precision in (0, 1):
        X, X64, res = solve_gpu(P, precision=precision)
        assert_certified(res)
        check_against_oracle(P, X64, oracle_solve(P))


def test_long_signals_rescore_from_global_memory():
    """n > 8192: the selection's re-score reads the residual and b from global memory (up to
    8192 floats of them are staged in shared memory), and the residual runs in nine row blocks."""
    P = synth.small_problem(8200, 2000, 6, 20, 60, rho=10, seed=8200, lam_frac=0.02)
    Xo = oracle_solve(P)
    for precision in (0, 1):
        X, X64, res = solve_gpu(P, precision=precision)
        assert_certified(res)
        check_against_oracle(P, X64, Xo)


def test_c2_subset_all_signals():
    P = synth.make_config("c2", p=48)
    X, X64, res = solve_gpu(P)
    assert_certified(res)
    Xo = oracle_solve(P)
    check_against_oracle(P, X, Xo)
    check_against_oracle(P, X64, Xo)


def test_c2_full_sampled():
    """Full batch, the configuration the benchmark times: a sample checked
    against the oracle signal by signal; every signal's certificate re-checked
    in FP64 by the oracle's independent certify()."""
    P = synth.make_config("c2")
    X, X64, res = solve_gpu(P)
    assert_certified(res)
    idx = np.random.default_rng(0).choice(P.p, size=12, replace=False)
    check_against_oracle(P, X64[idx], oracle_solve(P, idx), idx)
    for i in range(P.p):
        c = oracle.certify(P.At, P.B[i], float(P.lam[i]), X64[i])
        # rigorous: the FP64 re-check is below the tolerance and below the GPU's own bound
        # (up to the oracle's rounding, ~1e-13 relative)
        assert c["kkt"] <= TOL * (1 + 1e-9), (i, c)
        assert c["kkt"] <= res.stats["kkt"][i] * (1 + 1e-9) + 1e-12, (i, c, res.stats["kkt"][i])
        assert abs(c["objective"] - res.stats["objective"][i]) <= 1e-9 * c["objective"]
        # the GPU's gap uses a certified bound on ||A^T r||_inf for its dual point (feasible,
        # slightly more conservative than the exact maximum the oracle takes)
        assert abs(c["gap"] - res.stats["gap"][i]) <= 1e-9, (i, c, res.stats["gap"][i])


def test_lambda_above_max_and_zero_signal():
    P = synth.small_problem(128, 600, 4, 5, 10, rho=4, seed=2)
    lam = (np.abs(P.At.astype(np.float64) @ P.B.astype(np.float64).T).max(axis=0) * 1.001).astype(np.float32)
    B = P.B.copy()
    B[2] = 0.0
    Q = synth.Problem("edge", P.At, B, lam, 4)
    X, X64, res = solve_gpu(Q)
    assert_certified(res)
    assert np.all(X == 0)
    assert np.all(res.stats["outer_iters"] == 1)


def test_orthonormal_closed_form():
    rng = np.random.default_rng(5)
    Qm, _ = np.linalg.qr(rng.standard_normal((64, 64)))
    At = Qm.T.astype(np.float32).copy()
    B = rng.standard_normal((6, 64)).astype(np.float32)
    lam = (0.2 * np.abs(At.astype(np.float64) @ B.T.astype(np.float64)).max(axis=0)).astype(np.float32)
    P = synth.Problem("orth", At, B, lam, 8)
    X, X64, res = solve_gpu(P)
    assert_certified(res)
    for i in range(P.p):
        ref = ck.soft_threshold_orthonormal(At, B[i], float(lam[i]))
        np.testing.assert_allclose(X64[i], ref, atol=1e-6 * np.abs(ref).max())


def test_host_buffers_match_device_buffers():
    P = synth.small_problem(256, 1024, 10, 5, 20, rho=5, seed=11)
    Xd, X64d, _ = solve_gpu(P, reentry=1)
    Xh, X64h, resh = solve_gpu(P, host=True, reentry=1)
    assert_certified(resh)
    np.testing.assert_array_equal(Xd, Xh)


def test_deterministic_repeat():
    P = synth.small_problem(256, 2048, 20, 10, 30, rho=6, seed=12)
    # MPL_OPT_REENTRY = 1: the same bits on every run (the default re-entry may differ in
    # the last bits from run to run, certified either way)
    X1, _, _ = solve_gpu(P, reentry=1)
    X2, _, _ = solve_gpu(P, reentry=1)
    np.testing.assert_array_equal(X1, X2)


def test_reentry_modes_agree():
    """Re-entry as soon as a signal's finish is done (the default) and exactly two outer
    iterations later (MPL_OPT_REENTRY = 1) both certify every signal, with the same outer
    iteration counts, and their solutions agree to the certificate's accuracy."""
    P = synth.make_config("c2", p=64)
    X0, X64_0, r0 = solve_gpu(P, precision=1)
    X1, X64_1, r1 = solve_gpu(P, precision=1, reentry=1)
    assert_certified(r0)
    assert_certified(r1)
    np.testing.assert_array_equal(r0.stats["outer_iters"], r1.stats["outer_iters"])
    np.testing.assert_allclose(X64_0, X64_1, rtol=0, atol=1e-9 * np.abs(X64_1).max())
    idx = np.arange(0, P.p, 8)
    check_against_oracle(P, X64_0[idx], oracle_solve(P, idx), idx)
    torch = _torch()
    s = mpl.Solver(torch.from_numpy(P.At).cuda(), rho=P.rho)
    assert mpl.mpl_get_option(s.h, mpl.MPL_OPT_REENTRY) == 0
    with pytest.raises(mpl.MplError):
        s.set(mpl.MPL_OPT_REENTRY, 2)
    s.close()


def test_empty_batch_and_bad_lambda():
    torch = _torch()
    P = synth.small_problem(64, 128, 3, 2, 4, rho=2, seed=3)
    s = mpl.Solver(torch.from_numpy(P.At).cuda(), rho=2)
    Xt = torch.zeros((0, P.m), device="cuda")
    r = s.solve(torch.zeros((0, P.n), device="cuda"), torch.zeros(0, device="cuda"), Xt)
    assert r.status == mpl.MPL_OK
    lam = P.lam.copy()
    lam[1] = -1.0
    Xt = torch.zeros((P.p, P.m), device="cuda")
    r = s.solve(torch.from_numpy(P.B).cuda(), torch.from_numpy(lam).cuda(), Xt)
    assert r.status == mpl.MPL_ERR_NOT_CONVERGED
    assert r.stats["status"][1] == mpl.MPL_SIG_NONFINITE
    assert r.stats["status"][0] == mpl.MPL_SIG_CERTIFIED
    s.close()


def test_graph_replay_matches_direct_launches():
    """Captured-and-replayed outer iterations give the same solutions as
    direct launches (first solve captures, second replays)."""
    P = synth.make_config("c2", p=40)
    Xd, X64d, rd = solve_gpu(P, graph=0, reentry=1)
    torch = _torch()
    s = mpl.Solver(torch.from_numpy(P.At).cuda(), rho=P.rho, graph=1, reentry=1)
    B = torch.from_numpy(P.B).cuda()
    lam = torch.from_numpy(P.lam).cuda()
    for _ in range(3):
        X = torch.empty((P.p, P.m), dtype=torch.float32, device="cuda")
        r = s.solve(B, lam, X, TOL)
        torch.cuda.synchronize()
        assert_certified(r)
        np.testing.assert_array_equal(X.cpu().numpy(), Xd)
    s.close()
