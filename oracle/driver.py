"""Adaptive multilevel Monte Carlo driver -- FP64 oracle (TEST INFRASTRUCTURE ONLY).

Follows Sec. 5 of the paper step by step:

* estimator P = sum_l Y_l, the telescoping sum of Eq. (mlmc:ident), with Y_0 and Y_l from
  Eqs. (mlmc:Yzero) and (Yldef);
* the sample counts N_l come from estimated variances (the remark "Constructive Upper Bound":
  a cheap pre-processing step estimates the variances and an optimisation problem gives N_l).
  Minimising the cost sum N_l C_l subject to sum V_l / N_l = eps^2 / 2 gives
  N_l = ceil(2 eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k C_k));
* levels are added until the bias is below eps / sqrt(2), so that bias^2 + variance <= eps^2,
  the mean-square error of the Theorem in Sec. 5.  The bias of a level-L estimate is read from
  the weak rate alpha of condition 1 of that Theorem: E[P - P_L] ~ m_L / (M^alpha - 1).

Readings (the paper gives the shape, not the numbers): L starts at Lmin with N0 warm-up
samples per level; alpha and beta are least-squares slopes of log_M |m_l| and log_M V_l over
l = 1..L, floored at 1/2; a level is added when every level needs at most 1% more samples and
the bias test fails; the new level's variance is extrapolated as V_{L-1} / M^beta; for l >= 2
the variance and |mean| used in these formulas are floored at half the extrapolation from the
level below, so that a level whose sample happens to show zero variance is not starved.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import Problem, level_sums as _oracle_level_sums


def level_cost(level: int, M: int) -> float:
    """C_l: Euler--Maruyama steps of one level-l sample (fine + coarse), Sec. 3 cost model."""
    return 1.0 if level == 0 else float(M ** level + M ** (level - 1))


@dataclass
class Estimate:
    P: float
    eps: float
    L: int
    converged: bool
    N: list = field(default_factory=list)
    sums: list = field(default_factory=list)
    mean: list = field(default_factory=list)
    var: list = field(default_factory=list)
    cost: list = field(default_factory=list)
    alpha: float = 0.0
    beta: float = 0.0
    total_cost: float = 0.0
    rounds: int = 0


def _slope(ls, ys):
    A = np.vstack([np.asarray(ls, float), np.ones(len(ls))]).T
    return float(np.linalg.lstsq(A, np.asarray(ys, float), rcond=None)[0][0])


def _rates(m, V, M, L):
    tiny = 1e-300
    ls = list(range(1, L + 1))
    a = -_slope(ls, [math.log(max(abs(m[l]), tiny), M) for l in ls])
    b = -_slope(ls, [math.log(max(V[l], tiny), M) for l in ls])
    return max(a, 0.5), max(b, 0.5)


def _n_opt(V, C, eps):
    tot = sum(math.sqrt(v * c) for v, c in zip(V, C))
    return [math.ceil(2.0 / eps ** 2 * math.sqrt(v / c) * tot) for v, c in zip(V, C)]


def estimate(eps: float, p: Problem, seed: int, M: int = 4, Lmin: int = 2, Lmax: int = 8, N0: int = 10_000,
             stream: str = "fp64", level_sums=None) -> Estimate:
    """Adaptive MLMC estimate of E[h(X(T))] to root-mean-square accuracy eps."""
    if level_sums is None:
        def level_sums(l, first, n):
            return _oracle_level_sums(l, M, n, p, seed, first=first, stream=stream)
    L = Lmin
    Nl = [0] * (L + 1)
    S = [np.zeros(4) for _ in range(L + 1)]
    cost = [0.0] * (L + 1)
    dN = [N0] * (L + 1)
    alpha = beta = 0.5
    rounds = 0
    m = V = None
    while any(d > 0 for d in dN):
        rounds += 1
        for l in range(L + 1):
            if dN[l] > 0:
                s, c = level_sums(l, Nl[l], dN[l])
                S[l] = S[l] + s
                cost[l] += c
                Nl[l] += dN[l]
        m = [S[l][0] / Nl[l] for l in range(L + 1)]
        V = [max(S[l][1] / Nl[l] - m[l] ** 2, 0.0) for l in range(L + 1)]
        alpha, beta = _rates(m, V, M, L)
        mf, Vf = _floored(m, V, M, alpha, beta)
        C = [level_cost(l, M) for l in range(L + 1)]
        dN = [max(0, n - d) for n, d in zip(_n_opt(Vf, C, eps), Nl)]
        if all(d <= 0.01 * n for d, n in zip(dN, Nl)) and _bias(mf, M, alpha) > eps / math.sqrt(2) and L < Lmax:
            L += 1
            Vf.append(Vf[-1] / M ** beta)
            Nl.append(0)
            S.append(np.zeros(4))
            cost.append(0.0)
            C.append(level_cost(L, M))
            dN = [max(0, n - d) for n, d in zip(_n_opt(Vf, C, eps), Nl)]
    mf, _ = _floored(m, V, M, alpha, beta)
    converged = _bias(mf, M, alpha) <= eps / math.sqrt(2)
    return Estimate(P=float(sum(m)), eps=eps, L=L, converged=converged, N=list(Nl), sums=[list(x) for x in S],
                    mean=m, var=V, cost=cost, alpha=alpha, beta=beta, total_cost=float(sum(cost)), rounds=rounds)


def _floored(m, V, M, alpha, beta):
    mf, Vf = list(m), list(V)
    for l in range(2, len(m)):
        mf[l] = max(abs(mf[l]), 0.5 * abs(mf[l - 1]) / M ** alpha)
        Vf[l] = max(Vf[l], 0.5 * Vf[l - 1] / M ** beta)
    return mf, Vf


def _bias(mf, M, alpha):
    L = len(mf) - 1
    return max(abs(mf[L]), abs(mf[L - 1]) / M ** alpha) / (M ** alpha - 1.0)
