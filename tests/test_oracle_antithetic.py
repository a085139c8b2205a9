"""Pins of the oracle's antithetic level estimator (Sec. 7: antithetic variables inside multilevel
Monte Carlo, Giles and Szpruch): a second fine path takes each coarse step's M fine increments in
reverse order, the coarse path is shared, and Y = (P_f + P_f^a) / 2 - P_c."""
import math

import numpy as np
import pytest

import oracle
from oracle import Problem

GBM = dict(S0=100.0, r=0.05, sigma=0.2, T=1.0)


@pytest.mark.parametrize("M,level", [(2, 1), (2, 3), (4, 1), (4, 2), (8, 1)])
@pytest.mark.parametrize("payoff", ["asian", "lookback"])
def test_antithetic_sample_rebuilt_by_hand(M, level, payoff):
    """Euler--Maruyama paths rebuilt step by step from the sample's increments, the antithetic
    one from the increments reversed inside every coarse step; compared bit for bit."""
    p = Problem(payoff=payoff, **GBM)
    n = M ** level
    h = p.T / n
    Y = oracle.level_samples(level, M, 6, p, seed=41, mode=oracle.MODE_ANTITHETIC)
    for s in range(6):
        dW, fine, coarse = oracle.sample_paths(level, M, s, p, seed=41)
        anti = np.concatenate([dW[c * M:(c + 1) * M][::-1] for c in range(n // M)])
        X, path = p.S0, [p.S0]
        for i in range(n):
            X = X + p.r * X * h + p.sigma * X * anti[i]
            path.append(X)
        want = 0.5 * (oracle.payoff(p, fine) + oracle.payoff(p, np.array(path))) - oracle.payoff(p, coarse)
        assert Y[s] == want


@pytest.mark.parametrize("scheme", ["em", "milstein"])
def test_terminal_payoffs_do_not_change(scheme):
    """The step factors 1 + d commute, so the antithetic fine path ends where the fine path ends:
    for a payoff of S(T) alone Y is the coupled estimator's up to roundoff."""
    p = Problem(payoff="european", scheme=scheme, **GBM)
    for level in (1, 3):
        yc = oracle.level_samples(level, 4, 500, p, seed=8)
        ya = oracle.level_samples(level, 4, 500, p, seed=8, mode=oracle.MODE_ANTITHETIC)
        assert np.allclose(ya, yc, rtol=0, atol=1e-10)


def test_level0_is_the_plain_estimator():
    p = Problem(payoff="asian", **GBM)
    assert np.array_equal(oracle.level_samples(0, 4, 300, p, seed=2, mode=oracle.MODE_ANTITHETIC),
                          oracle.level_samples(0, 4, 300, p, seed=2))


@pytest.mark.parametrize("level", [1, 2, 3])
def test_unbiased_on_a_payoff_linear_in_the_average(level):
    """With K far below every path average the Asian payoff is e^{-rT} (A - K), and the exact
    Euler--Maruyama means E[S_i] = S0 (1 + r h)^i give E[Y_l] in closed form; the antithetic path
    has the law of the fine path, so the antithetic estimator has that mean too."""
    p = Problem(payoff="asian", K=-1000.0, **GBM)
    M, N = 4, 40000
    n = M ** level

    def mean_avg(steps):
        h = p.T / steps
        ES = p.S0 * (1 + p.r * h) ** np.arange(steps + 1)
        return np.mean(0.5 * (ES[:-1] + ES[1:]))

    exact = math.exp(-p.r * p.T) * (mean_avg(n) - mean_avg(n // M))
    y = oracle.level_samples(level, M, N, p, seed=12, mode=oracle.MODE_ANTITHETIC)
    assert abs(y.mean() - exact) < 4 * y.std() / math.sqrt(N) + 1e-12


@pytest.mark.parametrize("payoff,scheme,level,factor", [("asian", "em", 2, 3.0), ("asian", "milstein", 3, 30.0),
                                                        ("lookback", "em", 3, 1.5)])
def test_variance_reduction(payoff, scheme, level, factor):
    """The estimator's purpose: Var Y_l falls for path-dependent payoffs, most with Milstein
    (Sec. 7 remarks that the combination is particularly effective with Milstein)."""
    p = Problem(payoff=payoff, scheme=scheme, **GBM)
    yc = oracle.level_samples(level, 4, 20000, p, seed=3)
    ya = oracle.level_samples(level, 4, 20000, p, seed=3, mode=oracle.MODE_ANTITHETIC)
    assert yc.var() > factor * ya.var()


def test_cost_counts_both_fine_paths():
    p = Problem(payoff="asian", **GBM)
    _, cost = oracle.level_sums(2, 4, 100, p, seed=1, mode=oracle.MODE_ANTITHETIC)
    assert cost == 100 * (2 * 16 + 4)
