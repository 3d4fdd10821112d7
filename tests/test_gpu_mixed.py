"""Mixed precision (BF16 tensor-core correlation with FP32 re-scoring of the
candidate band) against the plain FP32 path and the FP64 oracle.

Selection ranks by the fixed-order FP32 re-score in both paths and the band
is rigorous, so the two paths pick the same atoms at every outer iteration
and produce bit-identical solutions."""
import numpy as np
import pytest

import oracle
from paper_1302_5010_gb300 import mpl, synth
from parity import check_against_oracle
from test_gpu_parity import assert_certified, oracle_solve, solve_gpu

pytestmark = pytest.mark.gpu


def test_mixed_c1():
    P = synth.make_config("c1")
    X, X64, res = solve_gpu(P, precision=1)
    assert_certified(res)
    check_against_oracle(P, X64, oracle_solve(P))


@pytest.mark.parametrize("n,m,p,rho", [(256, 1000, 37, 5), (1000, 2050, 21, 8)])
def test_mixed_ragged(n, m, p, rho):
    P = synth.small_problem(n, m, p, 5, min(40, n // 6), rho=rho, seed=3 * n + m + p, lam_frac=0.03)
    X, X64, res = solve_gpu(P, precision=1)
    assert_certified(res)
    check_against_oracle(P, X64, oracle_solve(P))


def test_mixed_identical_to_plain_c2():
    P = synth.make_config("c2", p=96)
    # (bit-for-bit comparisons run with the fixed re-entry of MPL_OPT_REENTRY = 1)
    Xp, X64p, rp = solve_gpu(P, precision=0, reentry=1)
    Xm, X64m, rm = solve_gpu(P, precision=1, reentry=1)
    assert_certified(rp)
    assert_certified(rm)
    np.testing.assert_array_equal(rp.stats["outer_iters"], rm.stats["outer_iters"])
    np.testing.assert_array_equal(rp.stats["active_size"], rm.stats["active_size"])
    np.testing.assert_array_equal(Xp, Xm)
    np.testing.assert_array_equal(X64p, X64m)
    idx = np.arange(0, P.p, 8)
    check_against_oracle(P, X64m[idx], oracle_solve(P, idx), idx)


@pytest.mark.parametrize("bn", [64, 256])
def test_gemm_tile_does_not_change_the_solution(bn):
    """The mixed path with another GEMM tile width solves to the same bits."""
    import torch
    P = synth.make_config("c5", p=24)
    At = torch.from_numpy(P.At).cuda()
    B, lam = torch.from_numpy(P.B).cuda(), torch.from_numpy(P.lam).cuda()
    out = []
    for tile in (128, bn):
        s = mpl.Solver(At, rho=P.rho, precision=1, smax=512, gemm_tile=tile, reentry=1)
        X = torch.empty((P.p, P.m), device="cuda")
        r = s.solve(B, lam, X)
        torch.cuda.synchronize()
        assert r.status == mpl.MPL_OK
        out.append((X.cpu().numpy(), r.stats["outer_iters"]))
        s.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
