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


@pytest.fixture()
def driver_mode(mlmc):
    prev = mlmc.mlmc_set_driver_mode("auto")
    yield mlmc
    mlmc.mlmc_set_driver_mode(prev)


@pytest.mark.parametrize("payoff,estimator,precision,eps,seed,Lmax", [
    ("asian", "coupled", "fp32", 1e-3, 1, 8), ("lookback", "coupled", "fp32", 3e-3, 2, 8),
    ("european", "coupled", "fp64", 1e-2, 3, 8), ("digital", "coupled", "fp32", 2e-3, 4, 8),
    ("asian", "antithetic", "fp32", 1e-3, 5, 8), ("lookback", "coupled", "fp32", 1e-3, 6, 5),
    ("asian", "coupled", "fp64_stream32", 3e-3, 7, 8)])
def test_device_rounds_equal_host_rounds(driver_mode, payoff, estimator, precision, eps, seed, Lmax):
    """The rounds run on the device (one graph launch: a driver kernel configures the level
    kernels by device-side graph updates) take the host driver's decisions: the same rounds,
    N_l and level sums, so the same estimate, bit for bit."""
    mlmc = driver_mode
    p = mlmc.Problem(payoff=payoff, estimator=estimator, **GBM)
    mlmc.mlmc_set_driver_mode("host")
    h = mlmc.mlmc_estimate(eps, p, seed, precision=precision, Lmax=Lmax)
    mlmc.mlmc_set_driver_mode("device")
    d = mlmc.mlmc_estimate(eps, p, seed, precision=precision, Lmax=Lmax)
    d2 = mlmc.mlmc_estimate(eps, p, seed, precision=precision, Lmax=Lmax)  # the cached graph, again
    assert not h.device_rounds and d.device_rounds and d2.device_rounds
    for x in (d, d2):
        assert x.N == h.N and x.L == h.L and x.rounds == h.rounds and x.converged == h.converged
        assert x.sums == h.sums and x.P == h.P and x.status == h.status
        assert x.alpha == pytest.approx(h.alpha, rel=1e-12) and x.beta == pytest.approx(h.beta, rel=1e-12)
        assert x.d2h_bytes > 0 and x.kernel_ms > 0


def test_device_rounds_match_oracle_driver(driver_mode):
    """The device driver's FP64 arithmetic takes the oracle driver's N_l schedule."""
    mlmc = driver_mode
    mlmc.mlmc_set_driver_mode("device")
    for payoff, eps, seed in (("european", 1e-2, 1), ("asian", 5e-3, 2)):
        p = mlmc.Problem(payoff=payoff, **GBM)
        est = mlmc.mlmc_estimate(eps, p, seed, precision="fp64")
        ref = oracle_driver.estimate(eps, oracle.Problem(payoff=payoff, Q=1.0,
                                                         **{k: v for k, v in GBM.items() if k != "cash"}), seed,
                                     stream="fp64")
        assert est.device_rounds
        assert est.N == ref.N and est.L == ref.L and est.converged == ref.converged
        assert abs(est.P - ref.P) <= 1e-12 * abs(ref.P)


def test_device_rounds_fall_back_for_other_models(driver_mode):
    """The quintic ODE keeps the host rounds: "auto" runs them there, "device" refuses, and the
    diverging explicit scheme still stops with MLMC_ENONFINITE."""
    mlmc = driver_mode
    q = mlmc.Problem(kind="quintic", scheme="tamed", payoff="second_moment", T=1.0)
    a = mlmc.mlmc_estimate(1e-2, q, 1)
    assert not a.device_rounds
    g = mlmc.mlmc_estimate(1e-2, mlmc.Problem(payoff="european", **GBM), 1)
    assert g.device_rounds
    mlmc.mlmc_set_driver_mode("device")
    with pytest.raises(mlmc.MLMCError) as ei:
        mlmc.mlmc_estimate(1e-2, q, 1)
    assert ei.value.status == mlmc.MLMC_ENOTIMPL
    with pytest.raises(mlmc.MLMCError):
        mlmc.mlmc_set_driver_mode(7)
    assert mlmc.mlmc_set_driver_mode("auto") == "device"
