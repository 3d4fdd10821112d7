"""Writes tiny_lasso.txt: a tiny LASSO instance and its exact minimiser.

The minimiser comes from brute-force enumeration of sign patterns
(oracle.checkers.bruteforce_lasso), i.e. from the optimality conditions of
eq. 2 checked on every candidate support, not from the MPL oracle under test.
Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
from oracle import checkers  # noqa: E402


def main():
    rng = np.random.Generator(np.random.PCG64(20130221))
    n, m = 6, 8
    At = rng.standard_normal((m, n))
    At /= np.linalg.norm(At, axis=1, keepdims=True)
    x0 = np.zeros(m)
    x0[[1, 4, 6]] = [1.5, -0.8, 0.6]
    b = At.T @ x0 + 0.01 * rng.standard_normal(n)
    lam = 0.05 * np.abs(At @ b).max()
    x = checkers.bruteforce_lasso(At, b, lam)
    with open(os.path.join(HERE, "tiny_lasso.txt"), "w") as f:
        f.write("# tiny LASSO instance (eq. 2): n m, then lambda, b (n), At (m rows of n), x* (m)\n")
        f.write("# x* by brute-force sign enumeration; written by make_golden.py\n")
        f.write(f"{n} {m}\n{lam:.17g}\n")
        f.write(" ".join(f"{v:.17g}" for v in b) + "\n")
        for j in range(m):
            f.write(" ".join(f"{v:.17g}" for v in At[j]) + "\n")
        f.write(" ".join(f"{v:.17g}" for v in x) + "\n")


if __name__ == "__main__":
    main()
