"""The QUINTIC_ODE level kernel (Sec. 5, Eq. count: dX = -X^5 dt, X(0) ~ N(0, 1), E[X(T)^2])
against the FP64 oracle on the identical random stream, and the driver on it.

Tolerances, from the arithmetic:
  * tamed steps: the step map x -> x + h f / (1 + h |f|) has slope in (0, 1] for h <= 1, so
    roundoff (a few roundings of relative size u per step) does not grow; over n steps it adds
    like a random walk.  X(0) carries the normal's error e_z (FP32: the hardware logarithm,
    square root, sine and cosine, below 2e-6 relative).  |X(T)| <= |X(0)|, so
    |Y_gpu - Y_oracle| <= 8 (1 + X0^2) (e_z + 4 u sqrt(n + 1)).
  * explicit steps on level 0 (one step X1 = X0 - X0^5): dY/dX0 = 2 X1 (1 - 5 X0^4), so
    |Y_gpu - Y_oracle| <= 16 (1 + |Y|) (e_z (1 + 5 X0^4) + 8 u).  Deeper explicit paths either
    stay small (checked like tamed ones) or blow up, where rounding differences are amplified
    without bound: those are checked to be large or non-finite on both sides.
"""
import math

import numpy as np
import pytest

from oracle import ode

from gpu_helpers import moment_sums, run_level

pytestmark = pytest.mark.gpu

U = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24}
EZ = {"fp64": 1e-15, "fp32": 2e-6}
T = 1.0


@pytest.fixture(scope="module")
def mlmc():
    from paper_1505_00965_gb300 import build

    build.build()
    from paper_1505_00965_gb300 import mlmc as binding

    return binding


def _problem(mlmc, scheme, estimator="coupled"):
    return mlmc.Problem(kind="quintic", scheme=scheme, payoff="second_moment", T=T, estimator=estimator)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("estimator", ["coupled", "single"])
@pytest.mark.parametrize("level,N,first", [(0, 20011, 3), (1, 20011, 977), (2, 8191, 5), (3, 4001, 2 ** 33 + 1),
                                           (5, 2001, 7), (6, 1001, 0)])
def test_tamed_samples_match_oracle(mlmc, level, N, first, estimator, precision):
    seed = 20240601
    p = _problem(mlmc, "tamed", estimator)
    sums, y = run_level(mlmc, level, 4, N, first, p, seed, precision)
    yo = ode.level_samples(level, 4, N, T, seed, "tamed", first=first, stream=precision,
                           fine_only=estimator == "single")
    x0 = ode.initial_values(level, first, N, seed, stream=precision)
    n = 4 ** level
    tol = 8.0 * (1.0 + x0 ** 2) * (EZ[precision] + 4 * U[precision] * math.sqrt(n + 1))
    assert np.all(np.abs(y - yo) <= tol)
    # the four sums against the device's own samples, and the mean against the oracle's
    own = moment_sums(y)
    scale = moment_sums(np.abs(y))
    assert np.all(np.abs(sums - own) <= 1e-6 * scale + 1e-12)
    assert abs(sums[0] / N - yo.mean()) <= np.mean(tol) + 1e-12 * np.abs(yo).mean()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_explicit_level0_matches_oracle(mlmc, precision):
    seed, N = 17, 30011
    p = _problem(mlmc, "em")
    _, y = run_level(mlmc, 0, 4, N, 11, p, seed, precision)
    yo = ode.level_samples(0, 4, N, T, seed, "em", first=11, stream=precision)
    x0 = ode.initial_values(0, 11, N, seed, stream=precision)
    tol = 16.0 * (1.0 + np.abs(yo)) * (EZ[precision] * (1.0 + 5.0 * x0 ** 4) + 8 * U[precision])
    assert np.all(np.abs(y - yo) <= tol)


def _amplification(x0, h, n):
    """Upper bound on how much the explicit map x -> x - h x^5 enlarges a perturbation over n
    steps from x0: the product of max(1, |1 - 5 h x_k^4|) along the path (first order)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    a = np.ones_like(x)
    with np.errstate(over="ignore", invalid="ignore"):
        for _ in range(n):
            a *= np.maximum(1.0, np.abs(1.0 - 5.0 * h * x ** 4))
            x = x - h * x ** 5
    return a


def test_explicit_deep_paths_match_or_blow_up_together(mlmc):
    """FP64, level 2 (16 steps): samples whose oracle path stays below 10 in size match to the
    tamed-style bound times the explicit map's amplification of a rounding difference along the
    path (near the blow-up threshold one step multiplies it by up to |1 - 5 h x^4|); the others
    are above 1e3 or non-finite on both sides."""
    seed, N = 23, 40000
    p = _problem(mlmc, "em")
    _, y = run_level(mlmc, 2, 4, N, 0, p, seed, "fp64")
    with np.errstate(over="ignore", invalid="ignore"):
        yo = ode.level_samples(2, 4, N, T, seed, "em", stream="fp64")
        x0 = ode.initial_values(2, 0, N, seed)
        xf = ode.path_end(x0, T / 16, 16, "em")
        xc = ode.path_end(x0, T / 4, 4, "em")
    calm = np.isfinite(xf) & np.isfinite(xc) & (np.abs(xf) < 10) & (np.abs(xc) < 10)
    wild = ~np.isfinite(yo) | (np.abs(yo) > 1e3)
    assert calm.sum() > 0.9 * N and wild.sum() > 50
    amp = np.maximum(_amplification(x0, T / 16, 16), _amplification(x0, T / 4, 4))
    tol = 8.0 * (1.0 + x0 ** 2) * (EZ["fp64"] + 4 * U["fp64"] * math.sqrt(17)) * amp
    assert np.all(np.abs(y[calm] - yo[calm]) <= 4.0 * tol[calm])
    assert np.all(~np.isfinite(y[wild]) | (np.abs(y[wild]) > 1e2))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_driver_stops_on_the_explicit_scheme_and_converges_tamed(mlmc, precision):
    """Sec. 5: multilevel Monte Carlo with explicit Euler--Maruyama diverges on Eq. (count); the
    driver reports non-finite level sums.  The tamed estimate reaches E[X(1)^2] within its
    accuracy plus the first-order bias allowance of the bias test."""
    with pytest.raises(mlmc.MLMCError) as ei:
        mlmc.mlmc_estimate(1e-3, _problem(mlmc, "em"), 1, precision=precision)
    assert ei.value.status == mlmc.MLMC_ENONFINITE
    exact = ode.exact_second_moment(T)
    for seed in (1, 2, 3):
        est = mlmc.mlmc_estimate(2e-3, _problem(mlmc, "tamed"), seed, precision=precision)
        assert est.converged
        assert abs(est.P - exact) < 3 * 2e-3, (seed, est.P, exact)
        # the fitted slopes include the pre-asymptotic level 1 (V_1 / V_2 is several hundred)
        assert est.beta > 1.5 and est.alpha > 0.7


def test_quintic_rejected_where_not_built(mlmc):
    p = _problem(mlmc, "tamed")
    with pytest.raises(mlmc.MLMCError) as ei:
        mlmc.mlmc_estimate_batch([(p, 1e-2, 1)])
    assert ei.value.status == mlmc.MLMC_ENOTIMPL
    with pytest.raises(mlmc.MLMCError) as ei:
        mlmc.mlmc_cv_create(4, p)
    assert ei.value.status == mlmc.MLMC_ENOTIMPL


@pytest.mark.parametrize("level,N,first", [(0, 3, 5), (0, 9, 6), (2, 1, 7), (4, 33, 2 ** 40 + 3)])
def test_tamed_ragged_ranges_and_fp64_on_fp32_stream(mlmc, level, N, first):
    """Ranges that start and end inside a Philox block of four samples, and FP64 arithmetic on
    the FP32 stream (the FP32 path's samples to the FP64 bound)."""
    seed = 9
    p = _problem(mlmc, "tamed")
    for precision, stream in (("fp64", "fp64"), ("fp64_stream32", "fp32")):
        _, y = run_level(mlmc, level, 4, N, first, p, seed, precision)
        yo = ode.level_samples(level, 4, N, T, seed, "tamed", first=first, stream=stream)
        x0 = ode.initial_values(level, first, N, seed, stream=stream)
        tol = 8.0 * (1.0 + x0 ** 2) * (EZ["fp64"] + 4 * U["fp64"] * math.sqrt(4 ** level + 1))
        assert np.all(np.abs(y - yo) <= tol), precision


def test_quintic_empty_range_and_noalloc(mlmc):
    """No samples give zero sums; the allocation-free entry point runs the quintic kernel too."""
    import torch

    p = _problem(mlmc, "tamed")
    sums, _ = run_level(mlmc, 2, 4, 0, 0, p, 1, "fp32")
    assert np.all(sums == 0)
    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    mlmc.mlmc_level_sums_noalloc(3, 4, 5000, 0, p, 1, d)
    torch.cuda.synchronize()
    ref, _ = run_level(mlmc, 3, 4, 5000, 0, p, 1, "fp32")
    np.testing.assert_allclose(d.cpu().numpy(), ref, rtol=1e-5)
