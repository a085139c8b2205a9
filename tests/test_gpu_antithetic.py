"""The antithetic level estimator on the GPU (Sec. 7: antithetic variables inside multilevel Monte
Carlo) against the FP64 oracle's antithetic mode on the identical random stream.

Y = (P_f + P_f^a) / 2 - P_c: the average of two fine payoffs, each within the per-sample bound of
the level parity tests, less the coarse payoff, so the same bound holds:
|Y_gpu - Y_oracle| <= 8 (u sqrt(n + 1) + e_z) S0 e^{rT}.
"""
import math

import numpy as np
import pytest

import oracle

from gpu_helpers import moment_sums, oracle_problem, run_level

pytestmark = pytest.mark.gpu

GBM = dict(S0=100.0, r=0.05, sigma=0.2, T=1.0, K=100.0, cash=1.0)
U = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24}
EZ = {"fp64": 1e-15, "fp32": 2e-6}
RTOL_MEAN = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def mlmc():
    from paper_1505_00965_gb300 import build

    build.build()
    from paper_1505_00965_gb300 import mlmc as binding

    return binding


def _bound(precision, level, M):
    return 8.0 * (U[precision] * math.sqrt(M ** level + 1) + EZ[precision]) * GBM["S0"] * math.exp(GBM["r"] * GBM["T"])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("scheme", ["em", "milstein"])
@pytest.mark.parametrize("payoff", ["asian", "lookback", "european", "geo_asian"])
@pytest.mark.parametrize("M,level,N,first", [(4, 0, 8001, 3), (4, 1, 8001, 977), (4, 2, 4001, 5), (4, 4, 2001, 2 ** 33),
                                             (4, 6, 301, 11), (2, 1, 8001, 1), (2, 3, 4001, 7), (2, 6, 1001, 0)])
def test_antithetic_samples_match_oracle(mlmc, M, level, N, first, payoff, scheme, precision):
    seed = 4242
    p = mlmc.Problem(payoff=payoff, scheme=scheme, estimator="antithetic", **GBM)
    op = oracle_problem(oracle, p)
    sums, y = run_level(mlmc, level, M, N, first, p, seed, precision)
    yo = oracle.level_samples(level, M, N, op, seed=seed, first=first, stream=precision, mode=oracle.MODE_ANTITHETIC)
    bound = _bound(precision, level, M)
    assert np.all(np.isfinite(y))
    assert np.max(np.abs(y - yo)) <= bound
    own, absy = moment_sums(y), np.abs(y)
    red_tol = 1e-12 if precision == "fp64" else 32 * U["fp32"]
    for k in range(4):
        assert abs(sums[k] - own[k]) <= red_tol * (np.sum(absy ** (k + 1)) + 1e-300), k
    fine = oracle.level_samples(level, M, N, op, seed=seed, first=first, stream=precision, mode=oracle.MODE_FINE_ONLY)
    sbar = max(np.mean(np.abs(fine)), 1e-300)
    assert abs(y.mean() - yo.mean()) <= RTOL_MEAN[precision] * max(abs(yo.mean()), sbar)


def test_cost_and_short_form(mlmc):
    p = mlmc.Problem(payoff="asian", estimator="antithetic", **GBM)
    sums, cost = mlmc.mlmc_level_sums_ex(3, 4, 1000, 0, p, 9)
    assert cost == 1000 * (2 * 64 + 16)
    _, y = run_level(mlmc, 3, 4, 1000, 0, p, 9, "fp32")
    np.testing.assert_allclose(sums, moment_sums(y), rtol=1e-5)


def test_antithetic_estimate_agrees_and_costs_less(mlmc):
    """Asian call with Milstein (where Sec. 7 expects the combination to be most effective):
    the antithetic estimate agrees with the coupled one within their accuracies, its level
    variances fall faster, and it needs less work to reach the same eps."""
    eps = 1e-3
    for seed in (1, 2):
        a = mlmc.mlmc_estimate(eps, mlmc.Problem(payoff="asian", scheme="milstein", estimator="antithetic", **GBM), seed)
        b = mlmc.mlmc_estimate(eps, mlmc.Problem(payoff="asian", scheme="milstein", **GBM), seed)
        assert a.converged and b.converged
        assert abs(a.P - b.P) < 3 * math.sqrt(2) * eps, (a.P, b.P)
        assert a.beta > b.beta
        assert a.total_cost < b.total_cost


def test_antithetic_rejections(mlmc):
    p = mlmc.Problem(payoff="asian", estimator="antithetic", **GBM)
    with pytest.raises(mlmc.MLMCError) as ei:
        mlmc.mlmc_level_sums_ex(3, 8, 100, 0, p, 1)
    assert ei.value.status == mlmc.MLMC_ENOTIMPL
    with pytest.raises(mlmc.MLMCError) as ei:
        mlmc.mlmc_level_sums_ex(5, 4, 100, 0, p, 1, launch={"lanes_per_path": 4})
    assert ei.value.status == mlmc.MLMC_EINVAL
    with pytest.raises(mlmc.MLMCError) as ei:
        mlmc.mlmc_estimate_batch([(p, 1e-2, 1)])
    assert ei.value.status == mlmc.MLMC_EINVAL


@pytest.mark.parametrize("level,N", [(1, 8001), (4, 1001)])
def test_antithetic_fp64_on_fp32_stream(mlmc, level, N):
    """FP64 arithmetic on the FP32 stream: the antithetic samples of the FP32 path, to the FP64
    bound against the oracle on that stream."""
    p = mlmc.Problem(payoff="asian", estimator="antithetic", **GBM)
    op = oracle_problem(oracle, p)
    _, y = run_level(mlmc, level, 4, N, 0, p, 21, "fp64_stream32")
    yo = oracle.level_samples(level, 4, N, op, seed=21, stream="fp32", mode=oracle.MODE_ANTITHETIC)
    assert np.max(np.abs(y - yo)) <= _bound("fp64", level, 4)


def test_antithetic_empty_and_ragged_ranges(mlmc):
    """No samples give zero sums; ranges that start and end inside a Philox block (level 0 packs
    four samples per block; M = 2 level 1 packs two) match the oracle sample for sample."""
    p = mlmc.Problem(payoff="lookback", estimator="antithetic", **GBM)
    sums, _ = run_level(mlmc, 3, 4, 0, 0, p, 1, "fp32")
    assert np.all(sums == 0)
    op = oracle_problem(oracle, p)
    for M, level, first, N in [(4, 0, 5, 3), (4, 0, 6, 9), (2, 1, 3, 4), (2, 1, 1, 1), (4, 2, 7, 1)]:
        _, y = run_level(mlmc, level, M, N, first, p, 3, "fp64")
        yo = oracle.level_samples(level, M, N, op, seed=3, first=first, stream="fp64", mode=oracle.MODE_ANTITHETIC)
        assert np.max(np.abs(y - yo)) <= _bound("fp64", level, M), (M, level, first, N)
