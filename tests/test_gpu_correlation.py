"""The worst-case analysis product g = A^T r (Algorithm 1) from both
correlation paths, against FP64 on the same data, within the rigorous error
bounds that the selection's candidate band relies on:

  FP32 SIMT path:   |c - a^T r| <= gamma_n * sum_k |a_k r_k|
  BF16 tensor path: |c - a16^T r16| <= n 2^-22 * sum_k |a16_k r16_k|   (accumulation)
                    |c - a^T r| <= (2^-7 + 2^-16 + n 2^-22) * ||a|| ||r||   (operands)
                    |c - a^T r| <= ||a - a16|| ||r|| + ||a16|| (||r - r16|| + n 2^-22 ||r16||)
                                                       (the measured form the selection uses)
"""
import numpy as np
import pytest

from paper_1302_5010_gb300 import mpl

pytestmark = pytest.mark.gpu

# (p <= 8 with n >= 256 takes the matrix-vector route, the others the GEMMs)
SHAPES = [(256, 1000, 1), (256, 1000, 37), (1000, 2050, 130), (1024, 8192, 256), (4096, 4096, 300),
          (1024, 40000, 3), (2048, 30000, 8), (1000, 20001, 5)]


def _bf16(x):
    """Round float32 to bfloat16 (round to nearest even) and back."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def _data(n, m, p, seed):
    rng = np.random.default_rng(seed)
    At = rng.standard_normal((m, n)).astype(np.float32)
    At /= np.linalg.norm(At, axis=1, keepdims=True)
    R = (rng.standard_normal((p, n)) * 0.3).astype(np.float32)
    return At, R


def _run(At, R, precision):
    import torch
    s = mpl.Solver(torch.from_numpy(At).cuda(), precision=precision)
    C = torch.empty((R.shape[0], At.shape[0]), dtype=torch.float32, device="cuda")
    s.correlate(torch.from_numpy(R).cuda(), C)
    torch.cuda.synchronize()
    s.close()
    return C.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n,m,p", SHAPES)
def test_fp32_path_within_gamma_n(n, m, p):
    At, R = _data(n, m, p, n + m + p)
    C = _run(At, R, 0)
    A64, R64 = At.astype(np.float64), R.astype(np.float64)
    exact = R64 @ A64.T
    absdot = np.abs(R64) @ np.abs(A64).T
    u = 2.0 ** -24
    gam = n * u / (1 - n * u)
    assert np.all(np.abs(C - exact) <= gam * absdot + 1e-30)


@pytest.mark.parametrize("n,m,p", SHAPES)
def test_bf16_path_within_bounds(n, m, p):
    At, R = _data(n, m, p, 7 * n + m + p)
    C = _run(At, R, 1)
    A16, R16 = _bf16(At).astype(np.float64), _bf16(R).astype(np.float64)
    exact16 = R16 @ A16.T
    absdot16 = np.abs(R16) @ np.abs(A16).T
    err16 = np.abs(C - exact16)
    assert np.all(err16 <= n * 2.0 ** -22 * absdot16 + 1e-30), err16.max()
    exact = R.astype(np.float64) @ At.astype(np.float64).T
    bound = (2.0 ** -7 + 2.0 ** -16 + n * 2.0 ** -22) * np.outer(np.linalg.norm(R, axis=1),
                                                                  np.linalg.norm(At, axis=1))
    assert np.all(np.abs(C - exact) <= bound)
    # and it is a real bf16 product, not a float32 one in disguise
    assert np.abs(C - exact).max() > 1e-6 * np.abs(exact).max()


@pytest.mark.parametrize("n,m,p", SHAPES)
def test_bf16_path_within_measured_bound(n, m, p):
    """The measured form, with the dictionary terms maximised over the atoms as the
    selection keeps them, holds for every score; it is far below the worst case."""
    At, R = _data(n, m, p, 11 * n + m + p)
    C = _run(At, R, 1)
    A64, R64 = At.astype(np.float64), R.astype(np.float64)
    A16, R16 = _bf16(At).astype(np.float64), _bf16(R).astype(np.float64)
    ea = np.linalg.norm(A64 - A16, axis=1).max()
    ta = np.linalg.norm(A16, axis=1).max()
    rn = np.linalg.norm(R64, axis=1)
    er = np.linalg.norm(R64 - R16, axis=1)
    tr = np.linalg.norm(R16, axis=1)
    bound = ea * rn + ta * (er + 1.25 * n * 2.0 ** -22 * tr)
    err = np.abs(C - R64 @ A64.T)
    assert np.all(err <= bound[:, None]), (err / bound[:, None]).max()
    worst = (2.0 ** -7 + 2.0 ** -16 + n * 2.0 ** -22) * rn * np.linalg.norm(A64, axis=1).max()
    assert np.all(bound < 0.6 * worst)


# More output tiles than the GPU has SMs: every persistent CTA of the tensor-core kernel
# takes several tiles, so the accumulator ping-pong (two TMEM accumulators), the phase flips
# of their full/empty barriers and the operand ring's wrap across tiles are all exercised.
MULTI_TILE = [(4096, 65536, 300), (1024, 65536, 1024), (2048, 32768, 512)]


@pytest.mark.parametrize("n,m,p", MULTI_TILE)
def test_bf16_persistent_multi_tile(n, m, p):
    At, R = _data(n, m, p, 13 * n + p)
    C = _run(At, R, 1)
    A16, R16 = _bf16(At).astype(np.float64), _bf16(R).astype(np.float64)
    exact16 = R16 @ A16.T
    absdot16 = np.abs(R16) @ np.abs(A16).T
    err16 = np.abs(C - exact16)
    assert np.all(err16 <= 1.25 * n * 2.0 ** -22 * absdot16 + 1e-30), (err16 / absdot16).max()
    # every element came from its own tile: a stale or swapped accumulator would be off by O(1)
    assert np.abs(C - exact16).max() <= 1e-3 * np.abs(exact16).max()


@pytest.mark.parametrize("n,m,p", MULTI_TILE[:1])
def test_fp32_multi_tile(n, m, p):
    At, R = _data(n, m, p, 17 * n + p)
    C = _run(At, R, 0)
    A64, R64 = At.astype(np.float64), R.astype(np.float64)
    u = 2.0 ** -24
    gam = n * u / (1 - n * u)
    assert np.all(np.abs(C - R64 @ A64.T) <= gam * (np.abs(R64) @ np.abs(A64).T) + 1e-30)


def _adversarial(kind, n, m, p, seed):
    """Operands where the tensor-core accumulation loses the most: every product of one sign,
    or one large product followed by many just below the accumulator's last kept bit."""
    rng = np.random.default_rng(seed)
    if kind == "equal_sign":
        At = np.abs(rng.standard_normal((m, n))).astype(np.float32)
        R = np.abs(rng.standard_normal((p, n))).astype(np.float32)
    elif kind == "equal_sign_wide_range":
        At = (np.abs(rng.standard_normal((m, n))) * 2.0 ** rng.integers(-12, 12, (m, n))).astype(np.float32)
        R = np.abs(rng.standard_normal((p, n))).astype(np.float32)
    elif kind == "head_and_tail":
        # r = 1 everywhere; a = (1, e, e, ...) with e = 1.5 2^-23 (exact in BF16): each small
        # product sits below 2^-22 of the running sum
        At = np.full((m, n), 1.5 * 2.0 ** -23, dtype=np.float32)
        At[:, 0] = 1.0
        At[:, 1:] *= (1.0 + rng.integers(0, 2, (m, n - 1))).astype(np.float32)  # 1.5 or 3 x 2^-23
        R = np.ones((p, n), dtype=np.float32)
    elif kind == "head_per_group":
        # one product of size 1 at the start of every group of 16 (one MMA's K), the others tiny
        At = np.full((m, n), 2.0 ** -13, dtype=np.float32)
        At[:, ::16] = 1.0
        R = np.ones((p, n), dtype=np.float32)
        R[:, 1::2] = 1.5
    else:
        raise ValueError(kind)
    At = _bf16(At)
    R = _bf16(R)
    return At, R


@pytest.mark.parametrize("kind", ["equal_sign", "equal_sign_wide_range", "head_and_tail", "head_per_group"])
@pytest.mark.parametrize("n", [4096, 16384])
def test_bf16_accumulator_assumption_adversarial(kind, n):
    """The BF16 path's error band assumes that the FP32 accumulation of the tensor cores
    loses at most 2^-22 of the running magnitude per added product, i.e. that
    |c - a^T r| <= 1.25 n 2^-22 sum_k |a_k r_k| for BF16 operands (their products are exact).
    This is an assumption about the hardware, not a documented guarantee; it is checked here
    at the benchmark's n = 4096 (and above) on data built to make truncation worst."""
    m, p = 1024, 256
    At, R = _adversarial(kind, n, m, p, n + len(kind))
    C = _run(At, R, 1)
    A64, R64 = At.astype(np.float64), R.astype(np.float64)
    exact = R64 @ A64.T
    absdot = np.abs(R64) @ np.abs(A64).T
    err = np.abs(C - exact)
    ratio = (err / (n * 2.0 ** -22 * absdot)).max()
    assert ratio <= 1.25, ratio


def _run_tile(At, R, bn):
    import torch
    s = mpl.Solver(torch.from_numpy(At).cuda(), precision=1, gemm_tile=bn)
    C = torch.empty((R.shape[0], At.shape[0]), dtype=torch.float32, device="cuda")
    s.correlate(torch.from_numpy(R).cuda(), C)
    torch.cuda.synchronize()
    s.close()
    return C.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("bn", [64, 256])
@pytest.mark.parametrize("n,m,p", [(4096, 65536, 300), (1000, 2050, 130), (256, 1000, 37)])
def test_bf16_tile_widths(bn, n, m, p):
    """The 64- and 256-signal tiles (their own TMA boxes, ring depths and TMEM accumulators)
    give the same scores as the 128-signal tile, bit for bit (the accumulation order along n
    does not depend on the tile), within the accumulation bound, on shapes with ragged tails
    and more tiles than SMs."""
    At, R = _data(n, m, p, 19 * n + p + bn)
    C = _run_tile(At, R, bn)
    C128 = _run_tile(At, R, 128)
    np.testing.assert_array_equal(C, C128)
    A16, R16 = _bf16(At).astype(np.float64), _bf16(R).astype(np.float64)
    err16 = np.abs(C - R16 @ A16.T)
    assert np.all(err16 <= 1.25 * n * 2.0 ** -22 * (np.abs(R16) @ np.abs(A16).T) + 1e-30)
