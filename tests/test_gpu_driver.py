"""The adaptive driver on the GPU (Sec. 5: telescoping estimator, N_l from estimated variances,
bias test): its per-level sums against single-pass recomputation, its FP64 schedule and
estimate against the oracle's driver, coverage over seeds, and the Lmax status."""
import math

import numpy as np
import pytest

import oracle
from oracle import driver as oracle_driver

from closed_forms import black_scholes_call, digital_call

pytestmark = pytest.mark.gpu

GBM = dict(S0=100.0, r=0.05, sigma=0.2, T=1.0, K=100.0, cash=1.0)


@pytest.fixture(scope="module")
def mlmc():
    from paper_1505_00965_gb300 import build

    build.build()
    from paper_1505_00965_gb300 import mlmc as binding

    return binding


@pytest.mark.parametrize("payoff,precision,eps,seed", [("european", "fp64", 1e-2, 1), ("asian", "fp32", 3e-3, 2),
                                                       ("lookback", "fp32", 1e-2, 2), ("digital", "fp64", 5e-3, 3)])
def test_driver_sums_equal_single_pass(mlmc, payoff, precision, eps, seed):
    """Rounds draw fresh samples by advancing `first`, so each level's accumulated sums are the
    sums of samples [0, N_l).  Recomputed in one launch, the level means agree within the level
    tolerance (1e-12 of the price scale in FP64, 1e-5 in FP32; a round may split deep paths over
    a different number of lanes, which changes FP32 roundoff but not the samples)."""
    p = mlmc.Problem(payoff=payoff, **GBM)
    est = mlmc.mlmc_estimate(eps, p, seed, precision=precision)
    assert est.rounds >= 2 and len(est.N) == est.L + 1
    rtol = 1e-12 if precision == "fp64" else 1e-5
    single = []
    for l, n in enumerate(est.N):
        s, cost = mlmc.mlmc_level_sums_ex(l, 4, n, 0, p, seed, precision=precision)
        single.append(s[0] / n)
        assert est.cost[l] == cost
    scale = abs(single[0])
    for l, n in enumerate(est.N):
        assert abs(est.sums[l][0] / n - single[l]) <= rtol * max(abs(single[l]), scale), (l, est.sums[l][0] / n,
                                                                                           single[l])
    assert est.P == pytest.approx(sum(est.mean), rel=1e-14)
    assert est.path_steps == sum(n * 4 ** l for l, n in enumerate(est.N))


def test_fp64_driver_matches_oracle_driver(mlmc):
    """Same stream, same reading of the algorithm: the FP64 GPU driver takes the oracle's N_l
    and its estimate agrees to 1e-12 of the price."""
    p = mlmc.Problem(payoff="european", **GBM)
    est = mlmc.mlmc_estimate(1e-2, p, 1, precision="fp64")
    ref = oracle_driver.estimate(1e-2, oracle.Problem(payoff="european", Q=1.0,
                                                      **{k: v for k, v in GBM.items() if k != "cash"}), 1,
                                 stream="fp64")
    assert est.N == ref.N and est.L == ref.L and est.converged == ref.converged
    assert abs(est.P - ref.P) <= 1e-12 * abs(ref.P)
    assert est.alpha == pytest.approx(ref.alpha, rel=1e-9) and est.beta == pytest.approx(ref.beta, rel=1e-9)


def test_fp32_estimates_cover_closed_forms(mlmc):
    """Theorem of Sec. 5: RMSE <= eps, so estimates stay within 3 eps of the exact price."""
    bs = black_scholes_call(100, 100, 0.05, 0.2, 1.0)
    errs = [mlmc.mlmc_estimate(1e-2, mlmc.Problem(payoff="european", **GBM), s).P - bs for s in range(1, 9)]
    assert max(abs(e) for e in errs) < 3e-2 and math.sqrt(np.mean(np.square(errs))) < 2e-2
    dg = digital_call(100, 100, 0.05, 0.2, 1.0)
    d = mlmc.mlmc_estimate(2e-3, mlmc.Problem(payoff="digital", **GBM), 1)
    assert abs(d.P - dg) < 3 * 2e-3


def test_lookback_reaches_lmax_and_reports_it(mlmc):
    """A discretely monitored maximum converges at weak order 1/2: the bias test cannot pass
    below Lmax = 4 at eps = 1e-2, and the driver says so while returning the estimate."""
    est = mlmc.mlmc_estimate(1e-2, mlmc.Problem(payoff="lookback", **GBM), 1, Lmax=4)
    assert est.status == mlmc.MLMC_ENOTCONV and not est.converged and est.L == 4
    assert 17.0 < est.P < 19.2


def test_estimates_repeat_exactly(mlmc):
    p = mlmc.Problem(payoff="asian", **GBM)
    a = mlmc.mlmc_estimate(3e-3, p, 5)
    b = mlmc.mlmc_estimate(3e-3, p, 5)
    assert a.P == b.P and a.N == b.N


def test_pooled_buffers_survive_shutdown_and_other_streams(mlmc):
    """The driver's device buffers are pooled between calls: estimates on another stream, after
    mlmc_shutdown released the pool, and after an interleaved estimate of another problem all
    repeat the first result exactly."""
    import torch

    p = mlmc.Problem(payoff="lookback", **GBM)
    a = mlmc.mlmc_estimate(1e-2, p, 3, Lmax=5)
    mlmc.mlmc_estimate(1e-2, mlmc.Problem(payoff="asian", **GBM), 4)
    b = mlmc.mlmc_estimate(1e-2, p, 3, Lmax=5)
    mlmc.mlmc_shutdown()
    c = mlmc.mlmc_estimate(1e-2, p, 3, Lmax=5)
    s = torch.cuda.Stream()
    d = mlmc.mlmc_estimate(1e-2, p, 3, Lmax=5, stream=s)
    torch.cuda.synchronize()
    for x in (b, c, d):
        assert x.P == a.P and x.N == a.N


def test_concurrent_estimates_on_two_streams(mlmc):
    """A round's launches spread over the caller's stream and the pooled set's own streams; two
    estimates running at once from two host threads on two streams (each with its own pooled
    set) give exactly their sequential results."""
    import threading

    import torch

    probs = [(mlmc.Problem(payoff="lookback", **GBM), 5), (mlmc.Problem(payoff="asian", **GBM), 6)]
    ref = [mlmc.mlmc_estimate(3e-3, p, s, Lmax=6) for p, s in probs]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    out = [None, None]

    def run(i):
        p, s = probs[i]
        out[i] = mlmc.mlmc_estimate(3e-3, p, s, Lmax=6, stream=streams[i])

    threads = [threading.Thread(target=run, args=(i,)) for i in range(2)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    torch.cuda.synchronize()
    for r, o in zip(ref, out):
        assert o is not None and o.P == r.P and o.N == r.N and o.sums == r.sums
