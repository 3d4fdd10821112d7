"""Learned warm start: the proposal network's hand-written training kernels
(finite-difference gradient check, decreasing loss) and its effect on the solve
(same certified solutions as a cold start, identical plain/mixed selections,
fewer outer iterations on held-out signals)."""
import numpy as np
import pytest

from paper_1302_5010_gb300 import mpl, synth
from parity import check_against_oracle
from test_gpu_parity import assert_certified, oracle_solve

pytestmark = pytest.mark.gpu
TOL = 1e-6


def _torch():
    import torch
    return torch


def _reference(P, precision=0):
    """GPU cold-start solutions (certified) used as training labels."""
    torch = _torch()
    s = mpl.Solver(torch.from_numpy(P.At).cuda(), rho=P.rho, precision=precision)
    X = torch.zeros((P.p, P.m), device="cuda")
    r = s.solve(torch.from_numpy(P.B).cuda(), torch.from_numpy(P.lam).cuda(), X, TOL)
    assert_certified(r)
    s.close()
    return X


def _trained(P_train, precision=0, epochs=4, candidates=64):
    torch = _torch()
    Xref = _reference(P_train, precision)
    s = mpl.Solver(torch.from_numpy(P_train.At).cuda(), rho=P_train.rho, precision=precision,
                   warm_candidates=candidates)
    losses = s.train_proposal(torch.from_numpy(P_train.B).cuda(), torch.from_numpy(P_train.lam).cuda(), Xref,
                              epochs=epochs)
    return s, losses


def test_gradient_matches_finite_differences():
    torch = _torch()
    P = synth.small_problem(256, 2048, 24, 8, 24, rho=6, seed=31)
    s, _ = _trained(P, epochs=1, candidates=32)
    Xref = _reference(P)
    B, lam = torch.from_numpy(P.B).cuda(), torch.from_numpy(P.lam).cuda()
    w0 = mpl.mpl_proposal_get_weights(s.h).astype(np.float64)
    loss0, g = mpl.mpl_proposal_loss_grad(s.h, B, P.p, lam, Xref)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(np.arange(6, 198), 4, replace=False),
                          rng.choice(np.arange(262, 4358), 8, replace=False), np.arange(4422, 4426), [4486]])
    for t in idx:
        eps = 2e-3 * max(1.0, abs(w0[t]))
        w = w0.copy(); w[t] += eps
        mpl.mpl_proposal_set_weights(s.h, w)
        lp, _ = mpl.mpl_proposal_loss_grad(s.h, B, P.p, lam, Xref)
        w[t] -= 2 * eps
        mpl.mpl_proposal_set_weights(s.h, w)
        lm, _ = mpl.mpl_proposal_loss_grad(s.h, B, P.p, lam, Xref)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[t]) <= 0.05 * abs(fd) + 2e-4, (t, fd, g[t])
    mpl.mpl_proposal_set_weights(s.h, w0)
    s.close()


def test_training_decreases_loss():
    P = synth.make_config("c2", p=384, seed_shift=9000)
    s, losses = _trained(P, epochs=6)
    assert losses[-1] < losses[0], losses
    s.close()


def test_warm_start_matches_cold_and_oracle():
    torch = _torch()
    s, _ = _trained(synth.make_config("c2", p=512, seed_shift=9000))
    P = synth.make_config("c2", p=40)
    B, lam = torch.from_numpy(P.B).cuda(), torch.from_numpy(P.lam).cuda()
    Xc = torch.zeros((P.p, P.m), device="cuda")
    rc = s.solve(B, lam, Xc, TOL)
    assert_certified(rc)
    s.set(mpl.MPL_OPT_WARM_START, 2)
    Xw = torch.zeros((P.p, P.m), device="cuda")
    rw = s.solve(B, lam, Xw, TOL)
    assert_certified(rw)
    idx = np.arange(0, P.p, 4)
    Xo = oracle_solve(P, idx)
    check_against_oracle(P, Xw.cpu().numpy()[idx], Xo, idx)
    check_against_oracle(P, Xw.cpu().numpy(), Xc.cpu().numpy().astype(np.float64))
    # the warm start saves outer iterations on held-out signals
    assert rw.stats["outer_iters"].mean() < rc.stats["outer_iters"].mean(), (
        rw.stats["outer_iters"].mean(), rc.stats["outer_iters"].mean())
    s.close()


def test_warm_start_plain_and_mixed_identical():
    torch = _torch()
    Ptr = synth.make_config("c2", p=256, seed_shift=9000)
    s0, _ = _trained(Ptr, precision=0)
    w = mpl.mpl_proposal_get_weights(s0.h)
    s1 = mpl.Solver(torch.from_numpy(Ptr.At).cuda(), rho=Ptr.rho, precision=1, warm_candidates=64)
    mpl.mpl_proposal_set_weights(s1.h, w)
    P = synth.make_config("c2", p=64)
    B, lam = torch.from_numpy(P.B).cuda(), torch.from_numpy(P.lam).cuda()
    out = []
    for s in (s0, s1):
        s.set(mpl.MPL_OPT_WARM_START, 2)
        s.set(mpl.MPL_OPT_REENTRY, 1)
        X = torch.zeros((P.p, P.m), device="cuda")
        r = s.solve(B, lam, X, TOL)
        assert_certified(r)
        out.append((X.cpu().numpy(), r.stats["outer_iters"]))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    s0.close()
    s1.close()
