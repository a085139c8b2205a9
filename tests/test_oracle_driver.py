"""Pins of the oracle's adaptive driver (Sec. 5: telescoping estimator, N_l from estimated
variances, bias test; the Theorem of Sec. 5 for the accuracy and cost claims)."""
import math

import numpy as np
import pytest

from oracle import Problem, driver

from closed_forms import black_scholes_call, digital_call, geometric_asian_call, lookback_fixed_call

GBM = dict(S0=100.0, r=0.05, sigma=0.2, T=1.0)


def test_level_cost_model():
    """Sec. 3: cost proportional to f, g evaluations; a coupled sample steps both grids."""
    assert driver.level_cost(0, 4) == 1
    assert driver.level_cost(1, 4) == 5
    assert driver.level_cost(3, 4) == 80
    assert driver.level_cost(2, 2) == 6


def test_nopt_formula_meets_variance_target():
    """N_l = ceil(2 eps^-2 sqrt(V_l/C_l) sum_k sqrt(V_k C_k)) gives sum V_l/N_l <= eps^2/2."""
    V = [40.0, 0.5, 0.12, 0.03]
    C = [driver.level_cost(l, 4) for l in range(4)]
    for eps in [1e-2, 3e-3]:
        N = driver._n_opt(V, C, eps)
        assert sum(v / n for v, n in zip(V, N)) <= eps ** 2 / 2 * (1 + 1e-12)
        # and it is the Lagrange optimum: N_l proportional to sqrt(V_l / C_l)
        r = [n / math.sqrt(v / c) for n, v, c in zip(N, V, C)]
        assert max(r) / min(r) < 1.001


@pytest.mark.parametrize("payoff,exact,tol_mult", [
    ("european", black_scholes_call(100, 100, 0.05, 0.2, 1.0), 3.0),
    ("digital", digital_call(100, 100, 0.05, 0.2, 1.0), 3.0),
    ("geo_asian", geometric_asian_call(100, 100, 0.05, 0.2, 1.0), 3.0),
])
def test_estimate_matches_closed_form(payoff, exact, tol_mult):
    """Theorem of Sec. 5: mean-square error below eps^2, so |P - exact| is a few eps at most."""
    eps = 2e-3 if payoff == "digital" else 1e-2
    est = driver.estimate(eps, Problem(payoff=payoff, **GBM), seed=3)
    assert est.converged
    assert abs(est.P - exact) < tol_mult * eps, (est.P, exact)


def test_lookback_estimate_below_continuous_price():
    """Discrete monitoring of the maximum lowers the price by about 0.5826 sigma sqrt(h) S0
    (a bias of order sqrt(h)), so the estimate sits below the continuous closed form."""
    est = driver.estimate(2e-2, Problem(payoff="lookback", **GBM), seed=4)
    cont = lookback_fixed_call(100, 100, 0.05, 0.2, 1.0)
    h = 1.0 / 4 ** est.L
    gap = cont - est.P
    assert -3 * 2e-2 < gap < 2.0 * 0.5826 * 0.2 * math.sqrt(h) * 100 + 3 * 2e-2, (est.P, cont, est.L)
    assert est.alpha < 0.9   # the weak rate of a discretely monitored maximum is about 1/2


def test_coverage_over_seeds():
    """Over eight seeds the European estimates at eps = 1e-2 stay within 3 eps of Black--Scholes
    and their root-mean-square error is of order eps."""
    exact = black_scholes_call(100, 100, 0.05, 0.2, 1.0)
    errs = [driver.estimate(1e-2, Problem(payoff="european", **GBM), seed=s).P - exact for s in range(1, 9)]
    assert max(abs(e) for e in errs) < 3e-2
    assert math.sqrt(np.mean(np.square(errs))) < 2e-2


def test_cost_scaling_eps2_log2():
    """Sec. 5: cost of order eps^-2 (log eps)^2 for Euler--Maruyama, so eps^2 * cost grows only
    slowly as eps falls (Fig. 3's observation), far below the eps^-1 growth of eps^2 * cost
    for standard Monte Carlo (Sec. 3)."""
    p = Problem(payoff="european", **GBM)
    c = {}
    for eps in [2e-2, 5e-3]:
        est = driver.estimate(eps, p, seed=6)
        c[eps] = eps ** 2 * est.total_cost
    ratio = c[5e-3] / c[2e-2]
    assert ratio < 3.0, c          # standard MC would give about 4 here
    assert ratio > 0.5, c


def test_driver_deterministic_and_levels_grow():
    p = Problem(payoff="asian", **GBM)
    a = driver.estimate(1e-2, p, seed=9)
    b = driver.estimate(1e-2, p, seed=9)
    assert a.P == b.P and a.N == b.N
    c = driver.estimate(2.5e-3, p, seed=9)
    assert c.L >= a.L
    assert all(n > 0 for n in c.N)
    # N_l decreases with l (more paths on the cheap levels, Fig. 3 upper-left)
    assert all(c.N[l] >= c.N[l + 1] for l in range(len(c.N) - 1))
