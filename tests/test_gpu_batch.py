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


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_chunks_match_oracle_per_sample(mlmc, precision):
    """One batched round (the batch kernel's chunk list, including split lanes on deep levels and
    the packed level-0 blocks) writes every sample's Y: each equals the oracle's sample on the
    identical stream within the per-sample bound of the level parity tests, and each task's sums
    are the sums of its own samples."""
    import torch

    import oracle

    from gpu_helpers import moment_sums, oracle_problem

    u, ez = (2.0 ** -24, 2e-6) if precision == "fp32" else (2.0 ** -53, 1e-15)
    specs = [("european", 0.2, 100.0, 0, 20011, 3), ("asian", 0.3, 95.0, 1, 4001, 977), ("lookback", 0.25, 105.0, 3, 1501, 7),
             ("digital", 0.2, 100.0, 4, 777, 2 ** 33 + 1), ("asian", 0.2, 100.0, 6, 301, 11),
             ("lookback", 0.4, 90.0, 7, 129, 0), ("european", 0.3, 110.0, 2, 0, 5), ("asian", 0.2, 100.0, 8, 33, 1)]
    tasks = [(mlmc.Problem(payoff=p, sigma=s, K=k, cash=1.0), 40 + i, l, first, N)
             for i, (p, s, k, l, N, first) in enumerate(specs)]
    total = sum(t[4] for t in tasks)
    d_y = torch.zeros(total, dtype=torch.float64, device="cuda")
    sums = mlmc.mlmc_level_sums_batch(tasks, precision=precision, d_y=d_y)
    y_all = d_y.cpu().numpy()
    off = 0
    for (prob, seed, level, first, N), s in zip(tasks, sums):
        y = y_all[off:off + N]
        off += N
        if N == 0:
            assert s == [0.0, 0.0, 0.0, 0.0]
            continue
        yo = oracle.level_samples(level, 4, N, oracle_problem(oracle, prob), seed=seed, first=first, stream=precision)
        bound = 8.0 * (u * math.sqrt(4 ** level + 1) + ez) * prob.S0 * math.exp(prob.r * prob.T)
        diff = np.abs(y - yo)
        if prob.payoff == "digital" and precision == "fp32":
            diff = diff[diff < 0.25 * prob.cash]  # threshold flips, checked in the level parity tests
        assert np.max(diff) <= bound, (prob.payoff, level, float(np.max(diff)), bound)
        own = moment_sums(y)
        tol = 1e-12 if precision == "fp64" else 32 * u
        for k in range(4):
            assert abs(s[k] - own[k]) <= tol * np.sum(np.abs(y) ** (k + 1)) + 1e-300, (level, k)
