"""Derive the residue background frequencies implied by BLOSUM62.

The protein workload draws residues i.i.d. from a background distribution p
and plants homologs whose substitutions follow P(b | a) proportional to
p_b * exp(lambda * s(a, b)).  No external frequency table is shipped, so p and
lambda are the ones the matrix itself implies: a log-odds matrix
s(a, b) = log(q_ab / (p_a p_b)) / lambda satisfies, for every a,

    sum_b p_b * exp(lambda * s(a, b)) = 1,        sum_a p_a = 1,  p > 0.

For a fixed lambda the first condition is the linear system
exp(lambda * S) p = 1; lambda is then the root of sum(p(lambda)) = 1.

Run as ``python -m workloads.derive_background`` to rewrite
``workloads/blosum62_background.txt``; the generator reads that file so that
every machine samples from the same numbers.
"""
from __future__ import annotations

import os

import numpy as np

from . import load_blosum62

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "blosum62_background.txt")


def implied_background(s: np.ndarray) -> tuple[float, np.ndarray]:
    s = s.astype(np.float64)

    def p_of(lam: float) -> np.ndarray:
        return np.linalg.solve(np.exp(lam * s), np.ones(s.shape[0]))

    def f(lam: float) -> float:
        return float(p_of(lam).sum() - 1.0)

    # sum(p) falls through 1 once; bracket it and bisect (plain, no scipy).
    lo, hi = 0.05, 2.0
    assert f(lo) > 0 > f(hi), "lambda bracket does not straddle the root"
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0:
            lo = mid
        else:
            hi = mid
    lam = 0.5 * (lo + hi)
    p = p_of(lam)
    p = p / p.sum()
    return lam, p


def main() -> None:
    s, names = load_blosum62()
    lam, p = implied_background(s)
    assert np.all(p > 0)
    with open(OUT, "w") as fh:
        fh.write("# Background frequencies implied by BLOSUM62 (written by "
                 "workloads/derive_background.py).\n")
        fh.write(f"lambda {lam:.17g}\n")
        for a, pa in zip(names, p):
            fh.write(f"{a} {pa:.17g}\n")
    print(f"lambda = {lam:.6f}; p = {np.round(p, 4)}")


if __name__ == "__main__":
    main()
