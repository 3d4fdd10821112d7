"""Subspace exploratory matching (Algorithm 2, MPL_OPT_OMEGA) on the GPU against
the FP64 oracle.

The GPU's master problems are FP32 and stop at eq. (inner), so the order of
|u| among the explored atoms may differ from the oracle's exact restricted
solutions when two are close; the path to the solution can then differ, but
the solution cannot (the LASSO minimiser is unique for these dictionaries).
What is unique is compared: the certified solution, and, on a dictionary where
the kept atom is decided by a wide margin, the atom that survives the first
iteration."""
import numpy as np
import pytest

from oracle import checkers as ck
from paper_1302_5010_gb300 import mpl, synth
from parity import check_against_oracle
from test_gpu_parity import assert_certified, oracle_solve, solve_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("omega", [2, 3])
def test_smpl_c2_subset(omega):
    P = synth.make_config("c2", p=64)
    Xp, X64p, rp = solve_gpu(P, precision=0, omega=omega, reentry=1)
    Xm, X64m, rm = solve_gpu(P, precision=1, omega=omega, reentry=1)
    assert_certified(rp)
    assert_certified(rm)
    # the re-score decides selection in both precisions: identical paths
    np.testing.assert_array_equal(Xp, Xm)
    np.testing.assert_array_equal(rp.stats["outer_iters"], rm.stats["outer_iters"])
    idx = np.arange(0, P.p, 6)
    check_against_oracle(P, X64m[idx], oracle_solve(P, idx), idx)


@pytest.mark.parametrize("n,m,p,rho,omega", [(256, 1000, 17, 5, 3), (198, 777, 9, 2, 4)])
def test_smpl_ragged_against_oracle(n, m, p, rho, omega):
    P = synth.small_problem(n, m, p, 4, min(30, n // 6), rho=rho, seed=11 * n + m, lam_frac=0.03)
    X, X64, res = solve_gpu(P, precision=0, omega=omega)
    assert_certified(res)
    check_against_oracle(P, X64, oracle_solve(P))


def _wedge():
    a1 = np.array([1.0, 0.0, 0.0])
    a3 = np.array([0.0, 1.0, 0.0])
    a2 = np.array([1.0, 1.0, 0.5])
    a2 /= np.linalg.norm(a2)
    a4 = np.array([0.3, -0.2, 1.0])
    a4 /= np.linalg.norm(a4)
    At = np.stack([a1, a2, a3, a4]).astype(np.float32)
    b = (At[0].astype(np.float64) + 0.9 * At[2]).astype(np.float32)
    return At, b


def _one_iteration(At, b, lam, omega):
    import torch
    s = mpl.Solver(torch.from_numpy(At).cuda(), rho=1, precision=0, omega=omega, max_outer=1)
    X = torch.zeros((1, At.shape[0]), device="cuda")
    s.solve(torch.from_numpy(b[None]).cuda(), torch.tensor([lam], dtype=torch.float32).cuda(), X)
    torch.cuda.synchronize()
    s.close()
    return X.cpu().numpy()[0]


def test_smpl_keeps_largest_restricted_coefficient():
    At, b = _wedge()
    lam = 0.05
    A64 = At.astype(np.float64)
    g = A64 @ b.astype(np.float64)
    order = sorted(range(4), key=lambda j: (-abs(g[j]), j))
    J = order[:3]
    u = ck.bruteforce_lasso(A64[J], b.astype(np.float64), lam)
    keep = J[int(np.argmax(np.abs(u)))]
    assert keep != order[0]
    x1 = _one_iteration(At, b, lam, 1)
    x3 = _one_iteration(At, b, lam, 3)
    assert np.flatnonzero(x1).tolist() == [order[0]]  # Algorithm 1 keeps the top correlation
    assert np.flatnonzero(x3).tolist() == [keep]      # Algorithm 2 keeps the largest |u|
