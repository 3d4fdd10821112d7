"""The allocation-free correlation entry point (mpl_correlate_noalloc).

It serves programs that own their device memory through their own pool and
cannot let a library call cudaMalloc behind their back.  The test calls it
through the C ABI twice in a row on caller-owned buffers and checks each result
against the handle-based mpl_correlate (same FP32 path) and against the
rounding-error bound of an FP32 dot product.  This file is collected last so a
failure here does not hide the rest of the suite; it also passes on its own in
a fresh process."""
import numpy as np
import pytest

from paper_1302_5010_gb300 import mpl

pytestmark = pytest.mark.gpu

SHAPES = [(250, 1000, 37), (1024, 8192, 256)]


def _data(n, m, p, seed):
    rng = np.random.default_rng(seed)
    At = rng.standard_normal((m, n)).astype(np.float32)
    At /= np.linalg.norm(At, axis=1, keepdims=True)
    R = (rng.standard_normal((p, n)) * 0.3).astype(np.float32)
    return At, R


@pytest.mark.parametrize("n,m,p", SHAPES)
def test_noalloc_matches_handle_path_twice(n, m, p):
    import torch
    At, R = _data(n, m, p, n + m)
    A_d = torch.from_numpy(At).cuda()
    R_d = torch.from_numpy(R).cuda()
    # reference: the existing entry point
    s = mpl.Solver(A_d, precision=0)
    C_ref = torch.empty((p, m), dtype=torch.float32, device="cuda")
    s.correlate(R_d, C_ref)
    s.close()
    ref = C_ref.cpu().numpy().astype(np.float64)
    exact = R.astype(np.float64) @ At.astype(np.float64).T
    u = 2.0 ** -24
    bound = (n * u / (1 - n * u)) * (np.abs(R).astype(np.float64) @ np.abs(At).astype(np.float64).T)
    for call in range(2):
        C = torch.full((p, m), float("nan"), dtype=torch.float32, device="cuda")
        rc = mpl.mpl_correlate_noalloc(A_d, n, m, R_d, p, C)
        assert rc == mpl.MPL_OK, (call, rc)
        torch.cuda.synchronize()
        got = C.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got)), call
        np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-7)
        assert np.all(np.abs(got - exact) <= bound + 1e-30), call


def test_noalloc_rejects_oversize_and_host_buffers():
    import torch
    At, R = _data(64, 128, 4, 1)
    A_d = torch.from_numpy(At).cuda()
    R_d = torch.from_numpy(R).cuda()
    C = torch.empty((4, 128), dtype=torch.float32, device="cuda")
    big = mpl.MPL_NOALLOC_MAX_SIGNALS + 1
    assert mpl.mpl_correlate_noalloc(A_d, 64, 128, R_d, big, C) == mpl.MPL_ERR_UNSUPPORTED
    assert mpl.mpl_correlate_noalloc(A_d, 64, 128, torch.from_numpy(R_d.cpu().numpy()).cuda(), 0, C) == mpl.MPL_OK


@pytest.mark.parametrize("case", ["host_A", "host_R", "host_C", "n_too_large", "m_too_large", "misaligned_A",
                                  "misaligned_R", "misaligned_C"])
def test_noalloc_refuses_before_any_launch(case):
    """Every argument check that guards the kernel's loads and stores returns MPL_ERR_ARG
    synchronously: host buffers, sizes outside the limits, and views whose start is not
    16-byte aligned (the kernel reads and writes float4 rows)."""
    import torch
    n, m, p = 64, 128, 4
    At, R = _data(n, m, p, 3)
    A_d = torch.from_numpy(At).cuda()
    R_d = torch.from_numpy(R).cuda()
    C = torch.zeros((p, m), dtype=torch.float32, device="cuda")
    # offset views one float into a larger allocation: contiguous, but 4-byte aligned only
    A_off = torch.zeros(m * n + 4, dtype=torch.float32, device="cuda")[1:1 + m * n]
    R_off = torch.zeros(p * n + 4, dtype=torch.float32, device="cuda")[1:1 + p * n]
    C_off = torch.zeros(p * m + 4, dtype=torch.float32, device="cuda")[1:1 + p * m]
    args = dict(A=A_d, n=n, m=m, R=R_d, C=C)
    if case == "host_A":
        args["A"] = At
    elif case == "host_R":
        args["R"] = R
    elif case == "host_C":
        args["C"] = np.zeros((p, m), dtype=np.float32)
    elif case == "n_too_large":
        args["n"] = 65537
    elif case == "m_too_large":
        args["m"] = (1 << 26) + 1
    elif case == "misaligned_A":
        args["A"] = A_off
    elif case == "misaligned_R":
        args["R"] = R_off
    elif case == "misaligned_C":
        args["C"] = C_off
    torch.cuda.synchronize()
    rc = mpl.mpl_correlate_noalloc(args["A"], args["n"], args["m"], args["R"], p, args["C"])
    assert rc == mpl.MPL_ERR_ARG, (case, rc)
    torch.cuda.synchronize()
    # nothing was written
    assert torch.count_nonzero(C).item() == 0
