"""Writes oracle_fp64_n2048.txt: reference values of the 2048-point FP64 workload (exponential
Matern, range 0.1, nugget 1e-6, tile 256, seed 1) computed by the CPU oracle alone -- the
log-determinant (Eq. 1), the log-likelihood of a seeded N(0, I) vector, and a few entries of L.
Run from the repository root: python tests/golden/make_oracle_golden.py"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2410_09819_gb300 import inputs  # noqa: E402

ENTRIES = [(0, 0), (1, 0), (255, 17), (256, 255), (1000, 999), (2047, 2046), (2047, 2047), (1500, 3)]


def values():
    w = inputs.WORKLOADS["fp64_n2048"]
    A = oracle.matern(w.points(), w.sigma2, w.range_a, w.nu, w.nugget)
    L = oracle.cholesky(A)
    y = inputs.gaussian(w.n, 1, seed=2)[:, 0]
    return {"logdet": oracle.logdet(L), "loglik": oracle.loglik(L, y),
            **{f"L[{i},{j}]": float(L[i, j]) for i, j in ENTRIES}}


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_fp64_n2048.txt")
    with open(out, "w") as f:
        f.write("# written by tests/golden/make_oracle_golden.py (CPU oracle only); y = gaussian(n, 1, seed=2)\n")
        for k, v in values().items():
            f.write(f"{k} {v!r}\n")
    print(out)
