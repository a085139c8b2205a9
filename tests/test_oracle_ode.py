"""Pins of the oracle for the non-globally-Lipschitz test problem of Sec. 5, Eq. (count):
dX = -X^5 dt, X(0) ~ N(0, 1), E[X(T)^2], with explicit and tamed Euler--Maruyama."""
import math

import numpy as np
import pytest

from oracle import ode


def test_exact_solution_solves_the_ode():
    """X(t) = X0 (1 + 4 t X0^4)^(-1/4) satisfies dX/dt = -X^5 (central differences) and X(0) = X0."""
    x0 = np.array([-2.5, -0.7, 0.1, 1.0, 3.0])
    assert np.array_equal(ode.exact_solution(x0, 0.0), x0)
    for t in (0.1, 0.5, 1.0):
        d = 1e-5
        dxdt = (ode.exact_solution(x0, t + d) - ode.exact_solution(x0, t - d)) / (2 * d)
        assert np.allclose(dxdt, -ode.exact_solution(x0, t) ** 5, rtol=1e-7, atol=1e-12)


def test_exact_second_moment_against_sampling():
    """The quadrature of E[X(T)^2] against the mean of X(T)^2 over 4 10^6 standard normal X0."""
    rng = np.random.default_rng(7)
    x0 = rng.standard_normal(4_000_000)
    v = ode.exact_solution(x0, 1.0) ** 2
    assert abs(ode.exact_second_moment(1.0) - v.mean()) < 4 * v.std() / math.sqrt(len(v))
    assert ode.exact_second_moment(0.0) == pytest.approx(1.0, abs=1e-10)


def test_tamed_scheme_converges_at_first_order():
    """Fixed X0: the tamed path's error at T = 1 falls by about 4 when the step falls by 4."""
    x0 = np.array([0.3, 1.0, 2.0])
    err = [np.abs(ode.path_end(x0, 1.0 / n, n, "tamed") - ode.exact_solution(x0, 1.0)) for n in (64, 256, 1024)]
    for a, b in zip(err, err[1:]):
        assert np.all((a / b > 3.0) & (a / b < 5.0))


def test_explicit_step_blows_up_as_computed_by_hand():
    """X0 = 2, h = 1/4: X1 = 2 - 32/4 = -6, X2 = -6 + 6^5/4 = 1938, and the path overflows within
    six steps; the tamed step from the same X0 shrinks towards 0."""
    x = np.array([2.0])
    assert ode.path_end(x, 0.25, 1, "em")[0] == -6.0
    assert ode.path_end(x, 0.25, 2, "em")[0] == 1938.0
    assert not np.isfinite(ode.path_end(x, 0.25, 6, "em")[0])
    t = [ode.path_end(x, 0.25, n, "tamed")[0] for n in range(1, 7)]
    assert all(0.0 < b < a for a, b in zip([2.0] + t, t))


def test_tamed_step_keeps_sign_and_never_grows():
    """For h <= 1 the tamed increment h f / (1 + h |f|) has the sign of -X and magnitude below
    min(1, |X|): 0 <= X_{n+1} / X_n <= 1."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal(100_000) * 3.0
    for h in (1.0, 0.25, 1e-3):
        y = ode.step(x, h, "tamed")
        ratio = y / x
        assert np.all((ratio >= 0.0) & (ratio <= 1.0))


def test_initial_values_are_standard_normal_and_shared_by_both_grids():
    x0 = ode.initial_values(3, 0, 40000, seed=11)
    assert abs(x0.mean()) < 5 / math.sqrt(len(x0))
    assert abs(x0.var() - 1.0) < 5 * math.sqrt(2 / len(x0))
    # Y = X_f^2 - X_c^2 with both paths from the same X0: X_f^2 - Y = X_c^2 <= X0^2 (tamed)
    Pf = ode.level_samples(3, 4, 4000, 1.0, 11, "tamed", first=123, fine_only=True)
    Y = ode.level_samples(3, 4, 4000, 1.0, 11, "tamed", first=123)
    Xc2 = Pf - Y
    x0 = ode.initial_values(3, 123, 4000, seed=11)
    assert np.all(Xc2 >= 0) and np.all(Xc2 <= x0 ** 2 * (1 + 1e-12))
    assert np.allclose(Xc2, ode.path_end(x0, 4.0 / 64, 16, "tamed") ** 2, rtol=1e-13, atol=1e-300)


def test_tamed_multilevel_rates_and_telescoping():
    """Weak order 1 (mean Y_l falls by about M) and strong order 1 (Var Y_l falls by about M^2)
    on levels 2..5; sum of the level means against the fine-only mean at L = 5."""
    M, N, T, seed = 4, 20000, 1.0, 5
    means, variances = [], []
    for l in range(6):
        Y = ode.level_samples(l, M, N, T, seed, "tamed")
        means.append(Y.mean())
        variances.append(Y.var())
    for l in range(2, 5):
        assert 2.5 < means[l] / means[l + 1] < 6.0, l
        assert 9.0 < variances[l] / variances[l + 1] < 25.0, l
    Pf = ode.level_samples(5, M, 200_000, T, seed + 1, "tamed", fine_only=True)
    se = math.sqrt(sum(v / N for v in variances) + Pf.var() / len(Pf))
    assert abs(sum(means) - Pf.mean()) < 4 * se
    # and both sit within the first-order bias of the exact value
    assert abs(Pf.mean() - ode.exact_second_moment(T)) < 4 * Pf.std() / math.sqrt(len(Pf)) + 4e-3


def test_initial_values_at_top_of_64_bit_sample_indices():
    """Sample indices up to 2^64 - 2: X(0) of sample s is normal (s mod 4) of Philox block
    floor(s / 4), including blocks the range covers only in part."""
    from oracle import normals

    first, N = 2 ** 64 - 7, 6
    x0 = ode.initial_values(3, first, N, 11, stream="fp32")
    blocks = {q: normals(11, 3, q, 4, stream="fp32") for q in (first // 4, (first + N - 1) // 4)}
    want = [blocks[s // 4][s % 4] for s in range(first, first + N)]
    np.testing.assert_array_equal(x0, want)
