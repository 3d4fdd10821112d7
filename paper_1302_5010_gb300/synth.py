"""Seeded synthetic batch sparse-recovery problems.

This module only draws inputs: dictionaries, sparse codes, signals and the
per-signal regularisation weights.  It contains none of the solver's
arithmetic, so both the FP64 CPU oracle and the CUDA path consume exactly the
same arrays.

Layouts (all C-contiguous numpy arrays):
  At      (m, n) float32  dictionary, atom-major: At[j] is atom a_j, i.e. the
                          column-major n x m matrix A of the paper (Sec. 1,
                          the measurement model b = A x + e).
  B       (p, n) float32  signals, B[i] = b_i (column-major n x p).
  lam     (p,)   float32  lambda_i, computed in float64 from the float32 data
                          and then rounded to float32, so both sides solve the
                          identical problem.
  X_true  (p, m) float64  the planted sparse codes (None where the workload
                          has no planted code).

Workloads follow the paper's two settings:
  * compressive sensing over Gaussian dictionaries with unit-norm atoms,
    Bernoulli- or Gaussian-valued sparse codes (Sec. 4.1, Sec. 5.1);
  * face recognition with a class-structured dictionary plus an identity
    block for occlusion (Sec. 1.1 and Sec. 5.2); the face datasets are stood
    in for by class subspaces, see ``face_problem``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class Problem:
    name: str
    At: np.ndarray
    B: np.ndarray
    lam: np.ndarray
    rho: int
    X_true: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.At.shape[1]

    @property
    def m(self) -> int:
        return self.At.shape[0]

    @property
    def p(self) -> int:
        return self.B.shape[0]

    def subset(self, idx) -> "Problem":
        idx = np.asarray(idx)
        return Problem(self.name + f"[{len(idx)}]", self.At, np.ascontiguousarray(self.B[idx]),
                       np.ascontiguousarray(self.lam[idx]), self.rho,
                       None if self.X_true is None else self.X_true[idx], dict(self.meta))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian_dictionary(n: int, m: int, seed: int) -> np.ndarray:
    """i.i.d. Gaussian atoms normalised to unit l2 norm, returned atom-major float32."""
    rng = _rng(seed)
    At = np.empty((m, n), dtype=np.float32)
    chunk = max(1, (1 << 24) // max(n, 1))
    for j0 in range(0, m, chunk):
        j1 = min(m, j0 + chunk)
        blk = rng.standard_normal((j1 - j0, n))
        blk /= np.linalg.norm(blk, axis=1, keepdims=True)
        At[j0:j1] = blk.astype(np.float32)
    return At


def lambdas_from_fraction(At: np.ndarray, B: np.ndarray, frac: float) -> np.ndarray:
    """lambda_i = frac * ||A^T b_i||_inf (the paper's parameterisation, Sec. 4.1),
    evaluated in float64 on the float32 data and rounded to float32."""
    p = B.shape[0]
    out = np.empty(p, dtype=np.float64)
    A64 = At.astype(np.float64)
    step = max(1, (1 << 26) // max(At.shape[0], 1))
    for i0 in range(0, p, step):
        i1 = min(p, i0 + step)
        G = A64 @ B[i0:i1].astype(np.float64).T
        out[i0:i1] = np.abs(G).max(axis=0)
    return (frac * out).astype(np.float32)


def sparse_codes(m: int, p: int, kmin: int, kmax: int, values: str, rng) -> np.ndarray:
    X = np.zeros((p, m), dtype=np.float64)
    for i in range(p):
        k = int(rng.integers(kmin, kmax + 1))
        supp = rng.choice(m, size=k, replace=False)
        if values == "gaussian":
            v = rng.standard_normal(k)
        elif values == "signed_uniform":  # +/-1 times U(0.5, 1.5)
            v = rng.choice([-1.0, 1.0], size=k) * rng.uniform(0.5, 1.5, size=k)
        elif values == "bernoulli":  # +/-1
            v = rng.choice([-1.0, 1.0], size=k)
        else:
            raise ValueError(values)
        X[i, supp] = v
    return X


def gaussian_problem(n: int, m: int, p: int, kmin: int, kmax: int, values: str, sigma: float,
                     lam_frac: float, rho: int, seed_A: int, seed_B: int, name: str = "gauss",
                     At: Optional[np.ndarray] = None, noise: str = "gaussian") -> Problem:
    """Compressive-sensing batch: b_i = A x_i + e_i with e_i ~ N(0, sigma^2 I), or with
    noise="uniform" e_i ~ U[-sigma, sigma]^n (the noise of the paper's Sec. 4 experiments)."""
    if At is None:
        At = gaussian_dictionary(n, m, seed_A)
    rng = _rng(seed_B)
    X = sparse_codes(m, p, kmin, kmax, values, rng)
    B = np.empty((p, n), dtype=np.float32)
    for i in range(p):
        nz = np.nonzero(X[i])[0]
        e = sigma * rng.standard_normal(n) if noise == "gaussian" else rng.uniform(-sigma, sigma, n)
        b = At[nz].astype(np.float64).T @ X[i, nz] + e
        B[i] = b.astype(np.float32)
    lam = lambdas_from_fraction(At, B, lam_frac)
    return Problem(name, At, B, lam, rho, X, dict(n=n, m=m, p=p, kmin=kmin, kmax=kmax, values=values,
                                                 sigma=sigma, noise=noise, lam_frac=lam_frac))


def big_dictionary_problem(n: int = 1024, m: int = 1 << 18, k: int = 150, rho: int = 20,
                           lam_frac: float = 0.005, seed: int = 0, p: int = 1) -> Problem:
    """The big-dictionary single-signal setting of the paper's Sec. 4.6 (there 2^12 x 2^20,
    k in 300..800), at the caller's size: Gaussian unit-norm atoms, a k-sparse code with
    N(0, 1) entries, noise U[-0.01, 0.01] (Sec. 4.1) and lambda = 0.005 ||A^T b||_inf."""
    return gaussian_problem(n, m, p, k, k, "gaussian", 0.01, lam_frac, rho, seed_A=30_000 + seed,
                            seed_B=40_000 + seed, name=f"bigdict{n}x{m}", noise="uniform")


def face_problem(n: int = 1024, classes: int = 100, per_class: int = 90, rank: int = 9,
                 p: int = 2048, noise: float = 0.05, corrupt: float = 0.10, lam_frac: float = 0.01,
                 rho: int = 10, seed_A: int = 1234 + 4, seed_B: int = 5678 + 4,
                 name: str = "face") -> Problem:
    """Face-recognition-shaped batch (Sec. 1.1, Sec. 5.2) with synthetic classes.

    Each class is a rank-``rank`` Gaussian subspace; a training "image" is a
    random point of it plus isotropic noise, shifted to be nonnegative and
    scaled to [0, 1] like pixel data, then normalised to a unit atom.  The
    dictionary is [D I], the identity absorbing occluded pixels.  A query is a
    fresh point of one class's subspace in the same pixel scale with a fraction
    ``corrupt`` of its pixels replaced by U(0, 1), normalised to unit norm.
    """
    rngA = _rng(seed_A)
    bases = rngA.standard_normal((classes, n, rank)) / np.sqrt(n)
    D = np.empty((classes * per_class, n), dtype=np.float64)
    for c in range(classes):
        W = rngA.standard_normal((rank, per_class))
        img = (bases[c] @ W).T + noise * rngA.standard_normal((per_class, n)) / np.sqrt(n)
        img -= img.min(axis=1, keepdims=True)
        img /= img.max(axis=1, keepdims=True)
        D[c * per_class:(c + 1) * per_class] = img / np.linalg.norm(img, axis=1, keepdims=True)
    At = np.concatenate([D, np.eye(n)], axis=0).astype(np.float32)
    rng = _rng(seed_B)
    B = np.empty((p, n), dtype=np.float32)
    label = np.empty(p, dtype=np.int64)
    ncor = int(round(corrupt * n))
    for i in range(p):
        c = int(rng.integers(classes))
        img = bases[c] @ rng.standard_normal(rank) + noise * rng.standard_normal(n) / np.sqrt(n)
        img -= img.min()
        img /= img.max()
        idx = rng.choice(n, size=ncor, replace=False)
        img[idx] = rng.uniform(0.0, 1.0, size=ncor)
        B[i] = (img / np.linalg.norm(img)).astype(np.float32)
        label[i] = c
    lam = lambdas_from_fraction(At, B, lam_frac)
    return Problem(name, At, B, lam, rho, None,
                   dict(n=n, m=At.shape[0], p=p, classes=classes, per_class=per_class,
                        rank=rank, corrupt=corrupt, lam_frac=lam_frac, label=label))


# The five workloads.  c1: single-signal MPL; c2: batch plain FP32 BMPL in the
# shape of the paper's Table I/II dictionary (2^10 x 2^13); c3: the large
# mixed-precision batch; c4: face-shaped [D I]; c5: streaming warm-start batches.
CONFIGS = {
    "c1": dict(kind="gauss", n=256, m=1024, p=1, kmin=10, kmax=10, values="gaussian",
               sigma=0.01, lam_frac=0.05, rho=2),
    "c2": dict(kind="gauss", n=1024, m=8192, p=256, kmin=20, kmax=60, values="signed_uniform",
               sigma=1e-3, lam_frac=0.02, rho=15),
    "c3": dict(kind="gauss", n=4096, m=65536, p=1024, kmin=100, kmax=400, values="gaussian",
               sigma=1e-3, lam_frac=0.01, rho=100),
    "c4": dict(kind="face", n=1024, p=2048, lam_frac=0.01, rho=10),
    "c5": dict(kind="gauss", n=2048, m=32768, p=4096, kmin=50, kmax=200, values="gaussian",
               sigma=1e-3, lam_frac=0.01, rho=50),
}
CONFIG_INDEX = {"c1": 1, "c2": 2, "c3": 3, "c4": 4, "c5": 5}


def make_config(name: str, p: Optional[int] = None, seed_shift: int = 0) -> Problem:
    """Build workload ``name`` (c1..c5).  ``p`` truncates the batch (the first
    p signals of the full stream are identical for any p); ``seed_shift``
    moves the signal seed only (disjoint training streams)."""
    cfg = dict(CONFIGS[name])
    idx = CONFIG_INDEX[name]
    seed_A, seed_B = 1234 + idx, 5678 + idx + seed_shift
    pp = cfg["p"] if p is None else int(p)
    if cfg["kind"] == "face":
        return face_problem(n=cfg["n"], p=pp, lam_frac=cfg["lam_frac"], rho=cfg["rho"],
                            seed_A=seed_A, seed_B=seed_B, name=name)
    return gaussian_problem(cfg["n"], cfg["m"], pp, cfg["kmin"], cfg["kmax"], cfg["values"],
                            cfg["sigma"], cfg["lam_frac"], cfg["rho"], seed_A, seed_B, name=name)


def small_problem(n: int, m: int, p: int, kmin: int, kmax: int, rho: int, lam_frac: float = 0.02,
                  values: str = "signed_uniform", sigma: float = 1e-3, seed: int = 7,
                  name: str = "small") -> Problem:
    """A reduced Gaussian workload for parity tests (sizes chosen by the caller)."""
    return gaussian_problem(n, m, p, kmin, kmax, values, sigma, lam_frac, rho,
                            seed_A=10_000 + seed, seed_B=20_000 + seed, name=name)


def big_dictionary_device(n: int = 4096, m: int = 1 << 20, k: int = 600, lam_frac: float = 0.005,
                          seed: int = 0, device: str = "cuda"):
    """The Sec. 4.6 setting at the paper's full size (2^12 x 2^20 atoms: 16 GiB in FP32),
    drawn on the device with torch's seeded Philox generator (a host draw of 4.3e9 normals
    takes minutes): Gaussian atoms normalised to unit norm, a k-sparse N(0, 1) code, noise
    U[-0.01, 0.01], lambda = lam_frac ||A^T b||_inf evaluated in float64 and rounded to
    float32.  Returns (At (m, n) float32, b (1, n) float32, lam (1,) float32, support (k,)
    int64, values (k,) float64) as device tensors."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(50_000 + seed)
    At = torch.empty((m, n), dtype=torch.float32, device=device)
    step = max(1, (1 << 28) // n)
    for j0 in range(0, m, step):
        blk = At[j0:j0 + step]
        blk.normal_(generator=g)
        blk /= torch.linalg.vector_norm(blk.double(), dim=1, keepdim=True).float()
    supp = torch.randperm(m, generator=g, device=device)[:k]
    vals = torch.randn(k, generator=g, device=device, dtype=torch.float64)
    e = (torch.rand(n, generator=g, device=device, dtype=torch.float64) * 2.0 - 1.0) * 0.01
    b64 = At[supp].double().T @ vals + e
    b = b64.float()
    amax = torch.zeros((), dtype=torch.float64, device=device)
    for j0 in range(0, m, step):
        amax = torch.maximum(amax, (At[j0:j0 + step].double() @ b.double()).abs().max())
    lam = (lam_frac * amax).float().reshape(1)
    return At, b.reshape(1, n), lam, supp, vals
