"""Batched adaptive estimates: many problems per round through one persistent kernel (each
problem still follows Sec. 5 on its own).  The batch must reproduce, problem by problem, the
sample sets and level means of single-problem computation."""
import math

import numpy as np
import pytest

from closed_forms import black_scholes_call, digital_call

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mlmc():
    from paper_1505_00965_gb300 import build

    build.build()
    from paper_1505_00965_gb300 import mlmc as binding

    return binding


@pytest.fixture(scope="module")
def workloads():
    from paper_1505_00965_gb300 import workloads as w

    return w


def test_fp64_batch_equals_single_estimates(mlmc):
    """In FP64 the batch's chunked sums agree with the per-level launches to rounding, so every
    problem takes the same N_l schedule as mlmc_estimate and lands on the same estimate."""
    probs = [(mlmc.Problem(payoff=p, sigma=s, K=k), 2e-2, seed)
             for seed, (p, s, k) in enumerate([("european", 0.2, 100.0), ("asian", 0.3, 95.0), ("digital", 0.25, 105.0),
                                               ("lookback", 0.2, 100.0), ("european", 0.4, 110.0)], start=1)]
    batch = mlmc.mlmc_estimate_batch(probs, precision="fp64", Lmax=5)
    for (prob, eps, seed), b in zip(probs, batch):
        single = mlmc.mlmc_estimate(eps, prob, seed, precision="fp64", Lmax=5)
        assert b.N == single.N and b.L == single.L and b.converged == single.converged
        assert abs(b.P - single.P) <= 1e-12 * max(abs(single.P), 1.0)


def test_batch_sums_equal_single_pass(mlmc, workloads):
    """Every problem's accumulated level sums are the sums of its samples [0, N_l): recomputed
    one level at a time they agree within the level tolerance (1e-5 of the price scale)."""
    qs = workloads.batch_problems(24, seed=7, eps_range=(5e-3, 2e-2))
    batch = mlmc.mlmc_estimate_batch(qs, Lmax=6)
    for q, b in zip(qs, batch):
        prob = mlmc.Problem(**{k: q[k] for k in ("S0", "r", "sigma", "T", "payoff", "K", "cash")})
        single = []
        for l, n in enumerate(b.N):
            s, _ = mlmc.mlmc_level_sums_ex(l, 4, n, 0, prob, q["seed"], precision="fp32")
            single.append(s[0] / n)
        scale = abs(single[0]) + 1e-3
        for l, n in enumerate(b.N):
            assert abs(b.sums[l][0] / n - single[l]) <= 1e-5 * max(abs(single[l]), scale), (q, l)
        assert b.P == pytest.approx(sum(b.mean), rel=1e-14)


def test_batch_estimates_match_closed_forms(mlmc):
    """European and digital problems of a batch land within 3 eps of their closed forms."""
    rng = np.random.default_rng(3)
    probs, exact = [], []
    for i in range(24):
        K, sigma, T = rng.uniform(85, 115), rng.uniform(0.15, 0.4), rng.uniform(0.5, 1.5)
        kind = "european" if i % 2 == 0 else "digital"
        prob = mlmc.Problem(payoff=kind, K=K, sigma=sigma, T=T)
        eps = 1e-2 if kind == "european" else 2e-3
        probs.append((prob, eps, 100 + i))
        exact.append(black_scholes_call(100, K, 0.05, sigma, T) if kind == "european"
                     else digital_call(100, K, 0.05, sigma, T))
    batch = mlmc.mlmc_estimate_batch(probs)
    for (prob, eps, _), b, ex in zip(probs, batch, exact):
        assert b.converged
        assert abs(b.P - ex) < 3 * eps, (prob, b.P, ex)


def test_batch_repeats_exactly_and_reports_lmax(mlmc, workloads):
    qs = workloads.batch_problems(16, seed=11, eps_range=(5e-3, 1e-2))
    a = mlmc.mlmc_estimate_batch(qs, Lmax=4)
    b = mlmc.mlmc_estimate_batch(qs, Lmax=4)
    assert [x.P for x in a] == [x.P for x in b]
    assert [x.N for x in a] == [x.N for x in b]
    for q, x in zip(qs, a):
        if not x.converged:
            assert x.L == 4 and x.status == mlmc.MLMC_ENOTCONV
        assert math.isfinite(x.P) and x.rounds >= 1
