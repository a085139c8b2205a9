"""Pins of the oracle's level estimator (Sec. 5: Eqs. mlmc:Dtl, mlmc:Yzero, Yldef, Fig. 2).

Each test ties the oracle to something other than itself: exact Euler--Maruyama moments,
closed-form option prices, the telescoping identity, the convergence orders of Sec. 2 and
Sec. 5, hand-evaluated payoffs, and a brute-force rebuild of the coarse path.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import Problem

from closed_forms import (black_scholes_call, central_moments_from_sums, em_linear_moments)

HERE = os.path.dirname(os.path.abspath(__file__))
GBM = dict(S0=100.0, r=0.05, sigma=0.2, T=1.0)


@pytest.mark.parametrize("stream", ["fp64", "fp32"])
@pytest.mark.parametrize("level,N", [(0, 200_000), (1, 200_000), (2, 100_000), (3, 40_000), (5, 4_000)])
def test_linear_payoff_matches_exact_em_moments(level, N, stream):
    """E[Y_l] and Var[Y_l] of the linear payoff have closed forms for Euler--Maruyama (Eq. em)
    on GBM; a dropped drift term, a wrong step size or a wrong coupling all move them."""
    p = Problem(payoff="linear", **GBM)
    sums, cost = oracle.level_sums(level, 4, N, p, seed=2024 + level, stream=stream)
    mean, var, mu4 = central_moments_from_sums(sums, N)
    EY, VY = em_linear_moments(level, 4, **GBM)
    se_mean = math.sqrt(VY / N)
    se_var = math.sqrt(max(mu4 - var ** 2, 0.0) / N)
    assert abs(mean - EY) < 4.5 * se_mean, (mean, EY, se_mean)
    assert abs(var - VY) < 4.5 * se_var, (var, VY, se_var)
    assert cost == N * (1 if level == 0 else 4 ** level + 4 ** (level - 1))


def test_level0_is_single_step_of_size_T():
    """Level 0 (Eq. mlmc:Yzero): one Euler--Maruyama step of size T, no coarse path."""
    p = Problem(payoff="linear", **GBM)
    dW, fine, coarse = oracle.sample_paths(0, 4, 17, p, seed=5)
    assert coarse is None and len(fine) == 2 and len(dW) == 1
    assert fine[1] == pytest.approx(100 * (1 + 0.05 * 1.0 + 0.2 * dW[0]), rel=1e-15)
    # and dW is sqrt(T) times the sample's normal: slot 17 mod 4 of block 17 div 4
    z = oracle.normals(5, 0, 17 // 4, 4)
    assert dW[0] == math.sqrt(1.0) * z[17 % 4]
    Y = oracle.level_samples(0, 4, 1, p, seed=5, first=17)
    assert Y[0] == fine[1]


@pytest.mark.parametrize("M,level", [(2, 1), (2, 3), (4, 1), (4, 2), (4, 3), (8, 1), (8, 2)])
def test_coarse_path_is_em_driven_by_summed_fine_increments(M, level):
    """Fig. 2: the coarse path is plain Euler--Maruyama with step M h driven by sums of M
    consecutive fine increments.  Rebuilt here step by step, compared bit for bit."""
    p = Problem(payoff="european", **GBM)
    for s in range(5):
        dW, fine, coarse = oracle.sample_paths(level, M, s, p, seed=99)
        n = M ** level
        h = p.T / n
        assert len(fine) == n + 1 and len(coarse) == n // M + 1
        X = p.S0
        for i in range(n):
            assert fine[i] == X
            X = X + p.r * X * h + p.sigma * X * dW[i]
        assert fine[n] == X
        X = p.S0
        for j in range(n // M):
            dWc = 0.0
            for q in range(M):
                dWc += dW[j * M + q]
            assert coarse[j] == X
            X = X + p.r * X * (M * h) + p.sigma * X * dWc
        assert coarse[-1] == X


def test_fine_increments_are_stream_normals():
    """Fine step k takes normal k of the sample, scaled by sqrt(h)."""
    p = Problem(payoff="european", **GBM)
    for level, M in [(0, 4), (1, 4), (2, 4), (3, 4), (1, 2), (4, 2), (1, 8)]:
        n = M ** level
        z = oracle.sample_normals(42, level, M, 7)
        dW, _, _ = oracle.sample_paths(level, M, 7, p, seed=42)
        np.testing.assert_array_equal(dW, math.sqrt(p.T / n) * z)


@pytest.mark.parametrize("M,level", [(4, 0), (4, 1), (4, 2), (4, 3), (2, 1), (2, 2), (2, 3), (2, 4), (8, 1)])
def test_grid_brownian_law(M, level):
    """The T/16 grid values are a Brownian path: Cov(W(s), W(t)) = min(s, t), on the levels whose
    grid is the fine path and on those refined by Brownian-bridge midpoints (a midpoint normal that
    reused one of the path's own would break the covariance); W(T) and the grid points the level's
    own grid contains equal the running sums of its fine increments."""
    T = 1.0
    n = 20000
    W = np.array([oracle.grid_brownian(level, M, s, T, seed=13) for s in range(n)])
    t = (np.arange(16) + 1) * T / 16
    cov = np.cov(W.T, bias=True)
    want = np.minimum.outer(t, t)
    assert np.max(np.abs(cov - want)) < 5 * math.sqrt(2.0 / n) * T
    assert np.max(np.abs(W.mean(axis=0))) < 5 * math.sqrt(T / n)
    p = Problem(payoff="european", T=T, **{k: v for k, v in GBM.items() if k != "T"})
    nf = M ** level
    for s in range(5):
        dW, _, _ = oracle.sample_paths(level, M, s, p, seed=13)
        Wg = oracle.grid_brownian(level, M, s, T, seed=13)
        cum = np.cumsum(dW)
        for k in range(nf):
            idx = (k + 1) * 16 // nf - 1 if nf <= 16 else None
            if idx is not None:
                assert Wg[idx] == pytest.approx(cum[k], rel=1e-13, abs=1e-14)
        assert Wg[15] == pytest.approx(cum[-1], rel=1e-12, abs=1e-14)


def test_payoffs_hand_evaluated():
    """Payoff definitions on a hand-made path S = (100, 105, 98, 110), r = 0.05, T = 1."""
    d = math.exp(-0.05)
    path = np.array([100.0, 105.0, 98.0, 110.0])
    want = {
        "european": d * 10.0,
        "asian": d * max((102.5 + 101.5 + 104.0) / 3 - 100.0, 0.0),
        "lookback": d * 10.0,
        "digital": d * 1.0,
        "linear": 110.0,
        "geo_asian": d * (math.exp((0.5 * (math.log(100) + math.log(105)) + 0.5 * (math.log(105) + math.log(98))
                                    + 0.5 * (math.log(98) + math.log(110))) / 3) - 100.0),
    }
    for name, v in want.items():
        got = oracle.payoff(Problem(payoff=name, K=100.0, Q=1.0, **GBM), path)
        assert got == pytest.approx(v, rel=1e-14), name
    # lookback includes S_0 in the maximum
    p = Problem(payoff="lookback", K=95.0, **GBM)
    assert oracle.payoff(p, np.array([100.0, 90.0, 92.0])) == pytest.approx(d * 5.0, rel=1e-14)


def test_sec6_payoff_cases_golden():
    """The discounted call and digital payoffs of Sec. 6, including h(100) = e^{-0.05T}(100+0)/2."""
    g = json.load(open(os.path.join(HERE, "golden", "sec6_workload.json")))
    for c in g["payoff_cases"]:
        p = Problem(payoff=c["payoff"], K=g["K"], Q=g["digital_cash"], **g["model"])
        want = eval(c["value_expr"], {"exp": math.exp})
        got = oracle.payoff(p, np.array([100.0, c["x"]]))
        assert got == pytest.approx(want, rel=1e-14, abs=0.0), c


def test_telescoping_identity():
    """Eq. (mlmc:ident): sum_l E[P_l - P_{l-1}] = E[P_L], with independent levels (Sec. 5)."""
    p = Problem(payoff="european", **GBM)
    L, N = 3, 60_000
    tel, var_tel = 0.0, 0.0
    for l in range(L + 1):
        s, _ = oracle.level_sums(l, 4, N, p, seed=31)
        m, v, _ = central_moments_from_sums(s, N)
        tel += m
        var_tel += v / N
    s, _ = oracle.level_sums(L, 4, N, p, seed=32, mode=oracle.MODE_FINE_ONLY)
    direct, v, _ = central_moments_from_sums(s, N)
    assert abs(tel - direct) < 4.5 * math.sqrt(var_tel + v / N)
    # and the fine-only level-L mean estimates the Euler--Maruyama price, which approaches
    # Black--Scholes at weak order one (Eq. emweak)
    assert abs(direct - black_scholes_call(100, 100, 0.05, 0.2, 1.0)) < 4.5 * math.sqrt(v / N) + 0.05


@pytest.mark.parametrize("payoff,beta_lo,beta_hi", [("european", 0.8, 1.25), ("asian", 0.8, 1.35),
                                                    ("lookback", 0.6, 1.2), ("digital", 0.3, 0.75)])
def test_variance_decay_rate(payoff, beta_lo, beta_hi):
    """Eq. (mlmc:varPlm1): V[Y_l] = O(dt_l) for Lipschitz payoffs, so log_M V_l falls with slope
    about -1 (beta ~ 1) once l is past the first few levels; the discontinuous digital payoff
    decays at about half that rate."""
    p = Problem(payoff=payoff, **GBM)
    ls = [3, 4, 5, 6]
    scale = 8 if payoff == "digital" else 1
    Ns = {3: 20_000 * scale, 4: 8_000 * scale, 5: 3_000 * scale, 6: 1_500 * scale}
    logv = []
    for l in ls:
        s, _ = oracle.level_sums(l, 4, Ns[l], p, seed=77)
        _, v, _ = central_moments_from_sums(s, Ns[l])
        logv.append(math.log(v, 4))
    beta = -np.polyfit(ls, logv, 1)[0]
    assert beta_lo < beta < beta_hi, beta


def test_weak_order_one_european():
    """Eq. (emweak): |E[P_l - P_{l-1}]| = O(dt_l), so the level means shrink by about M per level
    once past level 1 (whose coarse path is a single step of size T and sits outside the
    asymptotic regime: there the ratio is larger than M)."""
    p = Problem(payoff="european", **GBM)
    means = []
    for l, N in [(1, 400_000), (2, 300_000), (3, 500_000)]:
        s, _ = oracle.level_sums(l, 4, N, p, seed=5)
        means.append(s[0] / N)
    assert 2.5 < means[0] / means[1] < 11.0, means
    assert 2.0 < means[1] / means[2] < 8.0, means


def test_resume_from_offset_is_exact():
    """Samples are addressed by index, so [0, N) equals [0, a) + [a, N) sample by sample."""
    p = Problem(payoff="asian", **GBM)
    full = oracle.level_samples(3, 4, 300, p, seed=8)
    a = oracle.level_samples(3, 4, 120, p, seed=8)
    b = oracle.level_samples(3, 4, 180, p, seed=8, first=120)
    assert np.array_equal(full, np.concatenate([a, b]))


def test_invalid_arguments_rejected():
    p = Problem()
    with pytest.raises(ValueError):
        oracle.level_sums(-1, 4, 10, p, 1)
    with pytest.raises(ValueError):
        oracle.level_sums(2, 3, 10, p, 1)
    s, c = oracle.level_sums(2, 4, 0, p, 1)
    assert list(s) == [0, 0, 0, 0] and c == 0


@pytest.mark.parametrize("level,N", [(0, 200_000), (1, 200_000), (2, 100_000), (4, 10_000)])
def test_milstein_linear_payoff_matches_exact_moments(level, N):
    """Milstein (Sec. 5): E[Y_l] and Var[Y_l] of the linear payoff have closed forms."""
    from closed_forms import milstein_linear_moments

    p = Problem(payoff="linear", scheme="milstein", **GBM)
    sums, _ = oracle.level_sums(level, 4, N, p, seed=4242 + level)
    mean, var, mu4 = central_moments_from_sums(sums, N)
    EY, VY = milstein_linear_moments(level, 4, **GBM)
    assert abs(mean - EY) < 4.5 * math.sqrt(VY / N)
    assert abs(var - VY) < 4.5 * math.sqrt(max(mu4 - var ** 2, 0.0) / N)


def test_milstein_coarse_path_rebuilt_step_by_step():
    p = Problem(payoff="european", scheme="milstein", **GBM)
    dW, fine, coarse = oracle.sample_paths(2, 4, 3, p, seed=8)
    h = 1.0 / 16
    X = 100.0
    for j in range(4):
        dWc = 0.0
        for q in range(4):
            dWc += dW[4 * j + q]
        X = X + 0.05 * X * (4 * h) + 0.2 * X * dWc + 0.5 * 0.2 * 0.2 * X * (dWc * dWc - 4 * h)
        assert coarse[j + 1] == X


def test_milstein_variance_decays_twice_as_fast():
    """Strong order one of Milstein gives V_l = O(h_l^2) for a Lipschitz payoff: beta ~ 2
    (against ~1 for Euler--Maruyama), which puts MLMC in the eps^-2 regime of the Theorem."""
    p = Problem(payoff="european", scheme="milstein", **GBM)
    ls = [2, 3, 4, 5]
    Ns = {2: 40_000, 3: 20_000, 4: 8_000, 5: 4_000}
    logv = []
    for l in ls:
        s, _ = oracle.level_sums(l, 4, Ns[l], p, seed=31)
        _, v, _ = central_moments_from_sums(s, Ns[l])
        logv.append(math.log(v, 4))
    beta = -np.polyfit(ls, logv, 1)[0]
    assert 1.5 < beta < 2.6, beta
