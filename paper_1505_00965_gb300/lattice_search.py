"""Search for the Korobov multiplier of the control variate's lattice rule.

The mean of the learned control variate g over x ~ N(0, I_8) is estimated with randomly shifted
copies of the rank-1 lattice {frac(i z / n) : i = 0 .. n - 1}, z = (1, a, a^2, ..., a^7) mod n,
n = 2^16 (a Korobov lattice).  This script picks a: the odd multiplier (a unit mod 2^16) with the
smallest weighted P_2 figure of merit,

    P_2(z) = -1 + (1/n) sum_i prod_k (1 + gamma_k 2 pi^2 B_2(frac(i z_k / n))),
    B_2(t) = t^2 - t + 1/6,   gamma_k = k^-2,

the worst-case squared integration error over the unit ball of the weighted Korobov space of
smoothness 2 (Sloan and Joe, "Lattice Methods for Multiple Integration", 1994; Sloan and
Wozniakowski, J. Complexity 14, 1998, for the weights).  The weights decay along the inputs,
which are the path's increments in time order: a payoff that averages or tracks the path
depends less on each later increment.  Lattice points are exact integers i z_k mod n, so the
criterion is evaluated without rounding of the points.

    python -m paper_1505_00965_gb300.lattice_search [--n 65536] [--d 8]

prints the best multipliers.  Run once; the library carries the result as a constant.
"""
from __future__ import annotations

import argparse
import math

import numpy as np


def p2(n: int, z: np.ndarray) -> float:
    i = np.arange(n, dtype=np.int64)
    t = (np.outer(i, z) % n) / n
    gamma = 1.0 / np.arange(1, len(z) + 1, dtype=np.float64) ** 2
    return float(np.mean(np.prod(1.0 + gamma * 2.0 * math.pi ** 2 * (t * t - t + 1.0 / 6.0), axis=1)) - 1.0)


def korobov(n: int, a: int, d: int) -> np.ndarray:
    return np.array([pow(a, k, n) for k in range(d)], dtype=np.int64)


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n", type=int, default=65536)
    ap.add_argument("--d", type=int, default=8)
    ap.add_argument("--top", type=int, default=5)
    args = ap.parse_args(argv)
    n, d = args.n, args.d
    scores = []
    for a in range(3, n // 2, 2):   # a and n - a give the same lattice up to reflection
        scores.append((p2(n, korobov(n, a, d)), a))
    scores.sort()
    for s, a in scores[: args.top]:
        print(f"a = {a}: P_2 = {s:.6e}  z = {korobov(n, a, d).tolist()}")


if __name__ == "__main__":
    main()
