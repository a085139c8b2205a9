"""Seeded synthetic inputs (parameters only; none of the method's arithmetic).

The method's inputs are option problems: a GBM model, a payoff, an accuracy and a seed.
These generators produce the workloads the tests and benchmarks use, from a numpy seed.
"""
from __future__ import annotations

import numpy as np

PAYOFF_NAMES = ("european", "asian", "lookback", "digital")


def batch_problems(n: int = 512, seed: int = 12345, eps_range=(1e-3, 1e-2)) -> list[dict]:
    """n independent problems: K ~ U[80, 120], sigma ~ U[0.1, 0.5], T ~ U[0.25, 2], r = 0.05,
    S0 = 100, payoff uniform over European / Asian / lookback / digital (cash 1), eps
    log-uniform in eps_range, problem seeds 1..n."""
    rng = np.random.default_rng(seed)
    K = rng.uniform(80.0, 120.0, n)
    sigma = rng.uniform(0.1, 0.5, n)
    T = rng.uniform(0.25, 2.0, n)
    pay = rng.integers(0, len(PAYOFF_NAMES), n)
    lo, hi = np.log10(eps_range[0]), np.log10(eps_range[1])
    eps = 10.0 ** rng.uniform(lo, hi, n)
    return [dict(S0=100.0, r=0.05, sigma=float(sigma[i]), T=float(T[i]), payoff=PAYOFF_NAMES[pay[i]],
                 K=float(K[i]), cash=1.0, eps=float(eps[i]), seed=i + 1) for i in range(n)]
