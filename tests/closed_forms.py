"""Closed-form values that pin the oracle from outside (test helpers, no oracle code).

Each function is the textbook formula for geometric Brownian motion
dS = r S dt + sigma S dW (the asset model of Sec. 6 of the paper) or an exact moment of the
Euler--Maruyama recursion of Eq. (em) for that model.
"""
from __future__ import annotations

import math

from scipy.stats import norm


def black_scholes_call(S0, K, r, sigma, T):
    """E[e^{-rT} max(S_T - K, 0)] for exact GBM (the European call of Sec. 5 and Sec. 6)."""
    d1 = (math.log(S0 / K) + (r + 0.5 * sigma ** 2) * T) / (sigma * math.sqrt(T))
    d2 = d1 - sigma * math.sqrt(T)
    return S0 * norm.cdf(d1) - K * math.exp(-r * T) * norm.cdf(d2)


def digital_call(S0, K, r, sigma, T, Q=1.0):
    """E[e^{-rT} Q 1{S_T > K}] (the digital option of Sec. 6)."""
    d2 = (math.log(S0 / K) + (r - 0.5 * sigma ** 2) * T) / (sigma * math.sqrt(T))
    return Q * math.exp(-r * T) * norm.cdf(d2)


def geometric_asian_call(S0, K, r, sigma, T):
    """Continuous geometric average G = exp((1/T) int_0^T log S dt); log G is normal with mean
    log S0 + (r - sigma^2/2) T/2 and variance sigma^2 T / 3 (int_0^T W dt ~ N(0, T^3/3))."""
    mu = math.log(S0) + (r - 0.5 * sigma ** 2) * T / 2
    s = sigma * math.sqrt(T / 3.0)
    d2 = (mu - math.log(K)) / s
    d1 = d2 + s
    return math.exp(-r * T) * (math.exp(mu + 0.5 * s * s) * norm.cdf(d1) - K * norm.cdf(d2))


def lookback_fixed_call(S0, K, r, sigma, T):
    """Continuous-monitoring fixed-strike lookback call, running max starting at S0, K >= S0
    (reflection principle for the maximum of Brownian motion with drift)."""
    assert K >= S0
    sT = sigma * math.sqrt(T)
    d1 = (math.log(S0 / K) + (r + 0.5 * sigma ** 2) * T) / sT
    d2 = d1 - sT
    k = 2 * r / sigma ** 2
    return (S0 * norm.cdf(d1) - K * math.exp(-r * T) * norm.cdf(d2)
            + S0 * math.exp(-r * T) / k * (-(S0 / K) ** (-k) * norm.cdf(d1 - 2 * r * math.sqrt(T) / sigma)
                                          + math.exp(r * T) * norm.cdf(d1)))


def em_linear_moments(level, M, S0, r, sigma, T):
    """Exact E[Y_l] and Var[Y_l] for the undiscounted linear payoff P = S_N of Euler--Maruyama.

    Fine factors a_i = 1 + r h + sigma dW_i (dW_i iid N(0, h)), coarse factors
    b_j = 1 + r H + sigma (sum of the M fine dW in block j), H = M h.  Independence across
    steps gives E[S_N] = S0 (1 + r h)^n, E[S_N^2] = S0^2 ((1 + r h)^2 + sigma^2 h)^n and, per
    coarse block, E[prod a_i * b_j] = (1 + r h)^M (1 + r H) + M sigma^2 h (1 + r h)^(M-1).
    """
    n = M ** level
    h = T / n
    a = 1 + r * h
    Ef = S0 * a ** n
    Ef2 = S0 ** 2 * (a * a + sigma ** 2 * h) ** n
    if level == 0:
        return Ef, Ef2 - Ef ** 2
    nc = n // M
    H = M * h
    b = 1 + r * H
    Ec = S0 * b ** nc
    Ec2 = S0 ** 2 * (b * b + sigma ** 2 * H) ** nc
    Efc = S0 ** 2 * (a ** M * b + M * sigma ** 2 * h * a ** (M - 1)) ** nc
    EY = Ef - Ec
    EY2 = Ef2 - 2 * Efc + Ec2
    return EY, EY2 - EY ** 2


def central_moments_from_sums(sums, N):
    """(mean, variance, fourth central moment) from raw power sums sum Y^k, k = 1..4."""
    m1, m2, m3, m4 = (s / N for s in sums)
    var = m2 - m1 ** 2
    mu4 = m4 - 4 * m1 * m3 + 6 * m1 ** 2 * m2 - 3 * m1 ** 4
    return m1, var, mu4


def milstein_linear_moments(level, M, S0, r, sigma, T):
    """Exact E[Y_l] and Var[Y_l] of the linear payoff for the Milstein scheme on GBM:
    factors f = 1 + r h + sigma dW + sigma^2 (dW^2 - h) / 2.  E[f] = 1 + r h and
    E[f^2] = (1 + r h)^2 + sigma^2 h + sigma^4 h^2 / 2 (dW odd moments vanish, E[dW^4] = 3 h^2).
    Per coarse block (fine factors A_i, coarse factor B on the summed increment):
    E[prod A_i B] = (1 + r H) a^M + M sigma^2 h a^(M-1) + sigma^4 h^2 (M a^(M-1) + M (M-1) a^(M-2)) / 2,
    a = 1 + r h."""
    n = M ** level
    h = T / n
    a = 1 + r * h
    Ef = S0 * a ** n
    Ef2 = S0 ** 2 * (a * a + sigma ** 2 * h + 0.5 * sigma ** 4 * h * h) ** n
    if level == 0:
        return Ef, Ef2 - Ef ** 2
    nc = n // M
    H = M * h
    b = 1 + r * H
    Ec = S0 * b ** nc
    Ec2 = S0 ** 2 * (b * b + sigma ** 2 * H + 0.5 * sigma ** 4 * H * H) ** nc
    cross = (b * a ** M + M * sigma ** 2 * h * a ** (M - 1)
             + 0.5 * sigma ** 4 * h * h * (M * a ** (M - 1) + M * (M - 1) * a ** (M - 2)))
    Efc = S0 ** 2 * cross ** nc
    EY = Ef - Ec
    return EY, Ef2 - 2 * Efc + Ec2 - EY ** 2
