"""Parity of the CUDA level kernels with the FP64 CPU oracle on the identical random stream.

Both sides draw the same Philox4x32-10 words for every sample (the stream of include/mlmc.h),
so every sample's Y = P_l - P_{l-1} (Sec. 5, Eq. Yldef) is compared one by one, and the four
moment sums after them.

Tolerances (written from the arithmetic, u = unit roundoff of the path precision):
  * level means: |m_gpu - m_oracle| <= rtol * max(|m|, sbar) with rtol = 1e-12 (FP64 paths) and
    1e-5 (FP32 paths), the per-level mean tolerances set for this engine; sbar, the mean
    |P_l| of the level's fine payoffs, is the price scale the level means add up to.
  * per sample: each Euler--Maruyama step rounds once (relative u), the n = M^l roundings of a
    path add up like a random walk, and the normals carry the error of the logarithm, square
    root, sine and cosine (below 1e-15 in FP64; below 2e-6 for the FP32 hardware
    approximations).  |Y_gpu - Y_oracle| <= 8 (u sqrt(n + 1) + e_z) S0 e^{rT}.
  * higher moments follow from the per-sample bound: |d sum Y^k| <= k sum |Y|^{k-1} * bound.
  * digital payoff in FP32: a sample whose final value lies within the per-sample bound of K may
    land on the other side of K; such flips are listed, each is checked to lie within the bound,
    and the means are compared over the remaining samples.
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
PAYOFFS = ["european", "asian", "lookback", "digital", "linear", "geo_asian"]
# (level, N, first): several blocks and a ragged tail on every level, sized for the oracle
LEVELS_M4 = [(0, 20011, 0), (1, 20011, 977), (2, 8191, 5), (3, 4001, 123456789), (4, 3001, 7),
             (5, 1201, 2 ** 33 + 3), (6, 601, 11), (7, 257, 0)]


@pytest.fixture(scope="module")
def mlmc():
    from paper_1505_00965_gb300 import build

    build.build()
    from paper_1505_00965_gb300 import mlmc as binding

    return binding


def _bound(precision, level, M, p):
    n = M ** level
    return 8.0 * (U[precision] * math.sqrt(n + 1) + EZ[precision]) * p.S0 * math.exp(p.r * p.T)


def _check_level(mlmc, level, M, N, first, payoff, precision, launch=None, seed=20240601):
    p = mlmc.Problem(payoff=payoff, **GBM)
    op = oracle_problem(oracle, p)
    sums, y = run_level(mlmc, level, M, N, first, p, seed, precision, launch=launch)
    yo = oracle.level_samples(level, M, N, op, seed=seed, first=first, stream=precision)
    fine = oracle.level_samples(level, M, N, op, seed=seed, first=first, stream=precision,
                                mode=oracle.MODE_FINE_ONLY)
    sbar = max(np.mean(np.abs(fine)), 1e-300)
    bound = _bound(precision, level, M, p)
    diff = np.abs(y - yo)
    keep = np.ones(N, dtype=bool)
    if payoff == "digital" and precision == "fp32":
        flips = np.nonzero(diff > 0.25 * p.cash)[0]
        for i in flips:
            _, fpath, cpath = oracle.sample_paths(level, M, first + int(i), op, seed=seed, stream=precision)
            near = abs(fpath[-1] - p.K) <= bound or (cpath is not None and abs(cpath[-1] - p.K) <= bound)
            assert near, f"digital flip at sample {first + i} with S_n far from K"
        keep[flips] = False
        assert len(flips) <= max(2, N // 1000)
    assert np.all(np.isfinite(y))
    worst = float(diff[keep].max()) if keep.any() else 0.0
    assert worst <= bound, f"{payoff} {precision} l={level}: max |dY| = {worst:.3e} > {bound:.3e}"
    # the device's four sums against the same sums of the device's own Y (reduction check):
    # FP64 paths add in FP64; FP32 paths add batches of at most 32 samples in FP32 first,
    # a relative error of at most 32 u of the sum of |Y|^k
    own = moment_sums(y)
    absy = np.abs(y)
    red_tol = 1e-12 if precision == "fp64" else 32 * U["fp32"]
    for k in range(4):
        scale = np.sum(absy ** (k + 1)) + 1e-300
        assert abs(sums[k] - own[k]) <= red_tol * scale, (k, sums[k], own[k])
    # level mean and higher moments against the oracle
    m_gpu, m_orc = np.mean(y[keep]), np.mean(yo[keep])
    tol = RTOL_MEAN[precision] * max(abs(m_orc), sbar)
    assert abs(m_gpu - m_orc) <= tol, f"mean {m_gpu!r} vs {m_orc!r} (tol {tol:.3e})"
    # the same samples on both sides: the means differ by roundoff alone, which must stay far
    # below the level's statistical error (the relative bound above is loose on deep levels,
    # where m_l is small against the price scale)
    se = np.std(yo[keep], ddof=1) / math.sqrt(keep.sum()) if keep.sum() > 1 else 0.0
    if se > 0:
        assert abs(m_gpu - m_orc) <= 0.1 * se, f"mean error {abs(m_gpu - m_orc):.3e} against SE {se:.3e}"
    ref = moment_sums(yo[keep])
    got = moment_sums(y[keep])
    for k in range(1, 4):
        allowed = (k + 1) * np.sum(np.abs(yo[keep]) ** k) * bound + 1e-13 * abs(ref[k])
        assert abs(got[k] - ref[k]) <= allowed, (k, got[k], ref[k], allowed)
    return worst / bound


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("payoff", PAYOFFS)
@pytest.mark.parametrize("level,N,first", LEVELS_M4)
def test_level_matches_oracle_M4(mlmc, level, N, first, payoff, precision):
    _check_level(mlmc, level, 4, N, first, payoff, precision, launch={"lanes_per_path": 1})


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("payoff", ["european", "asian", "lookback", "geo_asian"])
@pytest.mark.parametrize("level,N,lanes", [(3, 1001, 4), (4, 1001, 8), (5, 601, 32), (6, 301, 16), (7, 129, 32)])
def test_split_lanes_match_oracle(mlmc, level, N, lanes, payoff, precision):
    """Time-parallel form: lanes of a warp split each path and join by a product scan."""
    _check_level(mlmc, level, 4, N, 31, payoff, precision, launch={"lanes_per_path": lanes, "threads_per_block": 128})


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("M,level,N,lanes", [(2, 1, 5001, 1), (2, 2, 5001, 1), (2, 3, 3001, 1), (2, 7, 999, 1),
                                             (2, 9, 301, 16), (8, 0, 4001, 1), (8, 1, 4001, 1), (8, 2, 2001, 1),
                                             (8, 4, 301, 1), (8, 4, 301, 32)])
@pytest.mark.parametrize("payoff", ["asian", "lookback", "linear"])
def test_other_refinement_factors(mlmc, M, level, N, lanes, payoff, precision):
    """Eq. (mlmc:Dtl) with M = 2 (the paper's example) and M = 8."""
    _check_level(mlmc, level, M, N, 3, payoff, precision, launch={"lanes_per_path": lanes})


@pytest.mark.parametrize("payoff", ["european", "asian", "lookback", "digital"])
@pytest.mark.parametrize("first,N", [(0, 20011), (3, 20013), (2 ** 34 - 4098, 20000)])
def test_level0_block_pairs_match_oracle(mlmc, payoff, first, N):
    """Level 0 on a grid of 2 blocks (512 threads): each thread runs its whole Philox blocks two
    at a time (the one-step call payoffs) and an unpaired last one alone, with partial blocks at
    the range's ends and, in the last case, Philox block index 2^32 (a span boundary of the
    loop's 32-bit offsets) inside the range."""
    _check_level(mlmc, 0, 4, N, first, payoff, "fp32", launch={"threads_per_block": 256, "blocks": 2})


@pytest.mark.parametrize("blocks", [0, 2])
@pytest.mark.parametrize("payoff", PAYOFFS)
@pytest.mark.parametrize("M,level,N,first", [(4, 1, 20011, 977), (4, 2, 8191, 5), (4, 3, 4001, 123456789),
                                             (4, 5, 1201, 2 ** 33 + 3), (4, 6, 601, 11), (4, 7, 257, 0),
                                             (2, 2, 5001, 3), (2, 5, 2001, 3), (8, 2, 2001, 3)])
def test_two_samples_per_thread_match_oracle(mlmc, M, level, N, first, payoff, blocks):
    """The two-samples-per-thread kernels (FP32 Euler--Maruyama, one thread per sample) step two
    samples in lockstep: every sample against the oracle.  On a grid of 2 blocks (512 threads) a
    thread runs pairs and then, where its last sample has no partner (N not a multiple of 1024),
    that sample alone; on the planner's grid most threads hold one sample and run it alone."""
    _check_level(mlmc, level, M, N, first, payoff, "fp32",
                 launch={"lanes_per_path": 1, "samples_per_thread": 2, "threads_per_block": 256, "blocks": blocks})


@pytest.mark.parametrize("threads,blocks,spt", [(32, 1, 2), (64, 3, 2), (512, 0, 2), (96, 5, 2)])
def test_two_samples_per_thread_launch_shapes(mlmc, threads, blocks, spt):
    """Grid strides of the two-sample loop: any grid gives the samples of the one-sample kernel,
    and sums equal to the sums of its own samples."""
    p = mlmc.Problem(payoff="lookback", **GBM)
    ref_sums, ref_y = run_level(mlmc, 3, 4, 5003, 1, p, 9, "fp32", launch={"samples_per_thread": 1})
    sums, y = run_level(mlmc, 3, 4, 5003, 1, p, 9, "fp32",
                        launch={"threads_per_block": threads, "blocks": blocks, "samples_per_thread": spt})
    assert np.max(np.abs(y - ref_y)) <= _bound("fp32", 3, 4, p)
    own = moment_sums(y)
    for k in range(4):
        assert abs(sums[k] - own[k]) <= 32 * U["fp32"] * np.sum(np.abs(y) ** (k + 1)), k


def test_two_samples_per_thread_rejected_where_not_built(mlmc):
    """samples_per_thread = 2 exists for FP32 Euler--Maruyama whole paths only."""
    import torch

    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    ws_bytes = mlmc.mlmc_level_workspace_bytes(3, 4, 100, "fp32", None)
    ws = torch.zeros(ws_bytes, dtype=torch.uint8, device="cuda")
    for prob, level, prec, launch in [
        (mlmc.Problem(payoff="asian", **GBM), 3, "fp64", {"samples_per_thread": 2}),
        (mlmc.Problem(payoff="asian", scheme="milstein", **GBM), 3, "fp32", {"samples_per_thread": 2}),
        (mlmc.Problem(payoff="asian", **GBM), 0, "fp32", {"samples_per_thread": 2}),
        (mlmc.Problem(payoff="asian", **GBM), 5, "fp32", {"samples_per_thread": 2, "lanes_per_path": 4}),
        (mlmc.Problem(payoff="asian", **GBM), 3, "fp32", {"samples_per_thread": 2, "threads_per_block": 1024}),
        (mlmc.Problem(payoff="asian", estimator="antithetic", **GBM), 3, "fp32", {"samples_per_thread": 2}),
        (mlmc.Problem(payoff="asian", **GBM), 3, "fp32", {"samples_per_thread": 3}),
    ]:
        with pytest.raises(mlmc.MLMCError) as ei:
            mlmc.mlmc_level_sums_async(level, 4, 100, 0, prob, 1, d, ws, ws_bytes, precision=prec, launch=launch)
        assert ei.value.status == mlmc.MLMC_EINVAL


@pytest.mark.parametrize("payoff", ["asian", "lookback", "digital"])
@pytest.mark.parametrize("level,N", [(0, 10_000_000), (1, 4_000_000)])
def test_fp32_presum_error_on_level_variance(mlmc, payoff, level, N):
    """FP32 paths add batches of at most 32 samples in FP32 before the FP64 sums.  The level
    variance V = S2/N - (S1/N)^2 from the device's sums against V from FP64 sums of the device's
    own samples: their difference is the pre-sum's error alone, at most
    32u (sum Y^2 + 2 |m| sum |Y|) / N, which cancellation amplifies by E[Y^2]/V relative to V
    (about 3.5 at level 0 of the Asian call); the test bounds it and requires it below 1e-5 of V."""
    p = mlmc.Problem(payoff=payoff, **GBM)
    sums, y = run_level(mlmc, level, 4, N, 0, p, 3, "fp32", launch={"lanes_per_path": 1})
    own = moment_sums(y)
    m_dev, m_own = sums[0] / N, own[0] / N
    v_dev, v_own = sums[1] / N - m_dev ** 2, own[1] / N - m_own ** 2
    bound = 32 * U["fp32"] * (own[1] + 2 * abs(m_own) * np.sum(np.abs(y))) / N
    assert abs(v_dev - v_own) <= bound, (v_dev, v_own, bound)
    assert abs(v_dev - v_own) <= 1e-5 * v_own, (v_dev, v_own)


@pytest.mark.parametrize("threads,blocks", [(32, 1), (64, 3), (1024, 0), (256, 7)])
def test_launch_shapes_agree(mlmc, threads, blocks):
    """Grid-stride loops and the two-stage reduction: any launch shape gives the same samples
    and sums equal to the sums of its own samples."""
    p = mlmc.Problem(payoff="asian", **GBM)
    ref_sums, ref_y = run_level(mlmc, 3, 4, 5003, 0, p, 9, "fp32")
    sums, y = run_level(mlmc, 3, 4, 5003, 0, p, 9, "fp32", launch={"threads_per_block": threads, "blocks": blocks})
    assert np.array_equal(y, ref_y)
    np.testing.assert_allclose(sums, ref_sums, rtol=1e-6)


def test_zero_samples_and_repeat_launches(mlmc):
    p = mlmc.Problem(payoff="european", **GBM)
    sums, _ = run_level(mlmc, 2, 4, 0, 0, p, 1, "fp32")
    assert list(sums) == [0, 0, 0, 0]
    a, ya = run_level(mlmc, 2, 4, 1000, 0, p, 1, "fp32")
    b, yb = run_level(mlmc, 2, 4, 1000, 0, p, 1, "fp32")
    assert np.array_equal(a, b) and np.array_equal(ya, yb)


def test_host_entry_points_agree_with_async(mlmc):
    p = mlmc.Problem(payoff="lookback", **GBM)
    sums_a, y = run_level(mlmc, 4, 4, 3000, 0, p, 1, "fp32")
    sums_b, cost = mlmc.mlmc_level_sums(4, 4, 3000, p, 1)
    np.testing.assert_allclose(sums_b, sums_a, rtol=1e-12)
    assert cost == 3000 * (256 + 64)
    sums_c, _ = mlmc.mlmc_level_sums_ex(4, 4, 3000, 0, p, 1, precision="fp32")
    np.testing.assert_allclose(sums_c, sums_a, rtol=1e-12)


def test_resume_offsets_compose(mlmc):
    """Samples are addressed by index: [0, N) = [0, a) + [a, N) sample by sample (Sec. 5's
    fresh samples per round come from advancing `first`)."""
    p = mlmc.Problem(payoff="asian", **GBM)
    _, y = run_level(mlmc, 5, 4, 900, 0, p, 4, "fp64")  # per-sample values are launch independent
    _, y1 = run_level(mlmc, 5, 4, 400, 0, p, 4, "fp64")
    _, y2 = run_level(mlmc, 5, 4, 500, 400, p, 4, "fp64")
    assert np.array_equal(y, np.concatenate([y1, y2]))


def test_config_plain_fp64_european_full(mlmc):
    """Plain MLMC in FP64: European call, M = 4, levels 0..4, N_l = 10^4, seed 1 -- the whole
    workload against the oracle, and the telescoped sum against Black--Scholes (10.4506)."""
    from closed_forms import black_scholes_call

    p = mlmc.Problem(payoff="european", **GBM)
    op = oracle_problem(oracle, p)
    total, var = 0.0, 0.0
    for level in range(5):
        sums, cost = mlmc.mlmc_level_sums_ex(level, 4, 10_000, 0, p, 1, precision="fp64")
        ref, ref_cost = oracle.level_sums(level, 4, 10_000, op, seed=1, stream="fp64")
        assert cost == ref_cost
        fine = oracle.level_samples(level, 4, 2000, op, seed=1, stream="fp64", mode=oracle.MODE_FINE_ONLY)
        sbar = np.mean(np.abs(fine))
        assert abs(sums[0] - ref[0]) / 1e4 <= 1e-12 * max(abs(ref[0]) / 1e4, sbar)
        np.testing.assert_allclose(sums[1], ref[1], rtol=1e-11)
        m = sums[0] / 1e4
        total += m
        var += (sums[1] / 1e4 - m * m) / 1e4
    bs = black_scholes_call(100, 100, 0.05, 0.2, 1.0)
    assert abs(total - bs) < 4 * math.sqrt(var) + 0.02


def test_workspace_reuse_across_grid_sizes(mlmc):
    """One workspace serves launches of any level and grid size in stream order (the adaptive
    driver reuses one): grids that shrink and grow give the sums of fresh workspaces."""
    import torch

    p = mlmc.Problem(payoff="lookback", **GBM)
    shapes = [(0, 400_003, 300), (1, 200_001, 7), (2, 50_001, 64), (0, 9_999, 1), (3, 20_001, 33), (1, 77_777, 129),
              (5, 3_001, 2)]
    ws_bytes = max(mlmc.mlmc_level_workspace_bytes(l, 4, n, "fp32", {"blocks": b}) for l, n, b in shapes)
    ws = torch.zeros(ws_bytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    outs = torch.zeros(len(shapes), 4, dtype=torch.float64, device="cuda")
    for i, (l, n, b) in enumerate(shapes):
        mlmc.mlmc_level_sums_async(l, 4, n, 11, p, 3, outs[i], ws, ws_bytes, precision="fp32",
                                   launch={"blocks": b}, stream=stream)
    torch.cuda.synchronize()
    for i, (l, n, b) in enumerate(shapes):
        ref, _ = run_level(mlmc, l, 4, n, 11, p, 3, "fp32", launch={"blocks": b})
        np.testing.assert_array_equal(outs[i].cpu().numpy(), ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("payoff", ["european", "asian", "lookback", "linear"])
@pytest.mark.parametrize("M,level,N,lanes", [(4, 0, 8001, 1), (4, 1, 6001, 1), (4, 3, 2001, 1), (4, 5, 601, 1),
                                             (4, 5, 301, 16), (2, 1, 4001, 1), (2, 4, 1001, 1), (8, 2, 1001, 1)])
def test_milstein_matches_oracle(mlmc, M, level, N, lanes, payoff, precision):
    """Milstein on both grids (Sec. 5): same stream, same per-sample bounds."""
    p = mlmc.Problem(payoff=payoff, scheme="milstein", **GBM)
    op = oracle_problem(oracle, p)
    sums, y = run_level(mlmc, level, M, N, 7, p, 11, precision, launch={"lanes_per_path": lanes})
    yo = oracle.level_samples(level, M, N, op, seed=11, first=7, stream=precision)
    assert np.max(np.abs(y - yo)) <= _bound(precision, level, M, p)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("level,lanes,spt", [(0, 1, 0), (2, 1, 0), (4, 1, 0), (5, 8, 0), (1, 1, 2), (4, 1, 2)])
def test_single_level_estimator_matches_oracle(mlmc, level, lanes, spt, precision):
    """The single-level estimator P_l (standard Monte Carlo, Sec. 3) against the oracle's
    fine-only mode (spt = 2: the two-samples-per-thread kernels, FP32 only)."""
    if spt == 2 and precision != "fp32":
        pytest.skip("two samples per thread: FP32 kernels")
    p = mlmc.Problem(payoff="asian", estimator="single", **GBM)
    op = oracle_problem(oracle, p)
    N = 1201
    sums, y = run_level(mlmc, level, 4, N, 3, p, 5, precision, launch={"lanes_per_path": lanes, "samples_per_thread": spt})
    yo = oracle.level_samples(level, 4, N, op, seed=5, first=3, stream=precision, mode=oracle.MODE_FINE_ONLY)
    assert np.max(np.abs(y - yo)) <= _bound(precision, level, 4, p)


@pytest.mark.parametrize("payoff", ["asian", "digital", "lookback"])
@pytest.mark.parametrize("level,N", [(0, 20011), (3, 3001), (6, 401)])
def test_fp64_on_fp32_stream(mlmc, payoff, level, N):
    """FP64 arithmetic on the FP32 stream draws the FP32 path's samples: it matches the FP64
    oracle on that stream to the FP64 bound, and the FP32 path differs from it by FP32 roundoff
    alone (the precision comparison at full size rests on this)."""
    p = mlmc.Problem(payoff=payoff, **GBM)
    op = oracle_problem(oracle, p)
    _, y64 = run_level(mlmc, level, 4, N, 0, p, 21, "fp64_stream32", launch={"lanes_per_path": 1})
    yo = oracle.level_samples(level, 4, N, op, seed=21, stream="fp32")
    assert np.max(np.abs(y64 - yo)) <= _bound("fp64", level, 4, p)
    _, y32 = run_level(mlmc, level, 4, N, 0, p, 21, "fp32", launch={"lanes_per_path": 1})
    d = np.abs(y32 - y64)
    if payoff == "digital":
        d = d[d < 0.25]  # threshold flips, checked in the level parity tests
    assert np.max(d) <= _bound("fp32", level, 4, p)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_level0_ranges_inside_one_philox_block(mlmc, precision):
    """Level 0 packs four samples per Philox block and runs the blocks wholly inside the range
    without range checks: ranges that start and end inside a block, or lie within one, match the
    oracle sample for sample."""
    p = mlmc.Problem(payoff="lookback", **GBM)
    op = oracle_problem(oracle, p)
    for first, N in [(5, 3), (6, 9), (1, 1), (3, 2), (7, 12), (4, 4), (2 ** 35 + 2, 7)]:
        sums, y = run_level(mlmc, 0, 4, N, first, p, 13, precision)
        yo = oracle.level_samples(0, 4, N, op, seed=13, first=first, stream=precision)
        assert np.max(np.abs(y - yo)) <= _bound(precision, 0, 4, p), (first, N)
        np.testing.assert_allclose(sums[0], y.sum(), rtol=1e-6)


@pytest.mark.parametrize("scheme,sigma", [("em", 4.0), ("milstein", 10.0)])
@pytest.mark.parametrize("lanes", [2, 8])
def test_split_lookback_with_sign_changes(mlmc, lanes, scheme, sigma):
    """Level 3 (h = 1/64).  Euler--Maruyama with sigma = 4: a step factor 1 + d is negative
    whenever the normal is below -2.  Milstein with sigma = 10: the factor's least value
    1/2 + r h - sigma^2 h / 2 is below zero.  Paths change sign and chunks of split paths start
    below zero, so the kernel that keeps each chunk's running minimum must be the one chosen: the
    maximum of a chunk that starts negative is its start times the chunk's relative minimum.
    FP64 paths (near-zero factors amplify FP32 rounding beyond the per-sample bound)."""
    p = mlmc.Problem(payoff="lookback", scheme=scheme, S0=100.0, r=0.05, sigma=sigma, T=1.0, K=100.0, cash=1.0)
    op = oracle_problem(oracle, p)
    level, M, N, seed = 3, 4, 2001, 8
    _, y = run_level(mlmc, level, M, N, 0, p, seed, "fp64", launch={"lanes_per_path": lanes})
    yo = oracle.level_samples(level, M, N, op, seed=seed, stream="fp64")
    flips = 0
    for s in range(200):
        _, fine, _ = oracle.sample_paths(level, M, s, op, seed=seed, stream="fp64")
        flips += int(np.any(fine < 0))
    assert flips > 20, flips  # the regime is the one described
    # Y is a difference of fine and coarse payoffs that reach 1e5: the bound scales with them
    fine = oracle.level_samples(level, M, N, op, seed=seed, stream="fp64", mode=oracle.MODE_FINE_ONLY)
    scale = 1.0 + np.abs(fine) + np.abs(fine - yo)
    assert np.max(np.abs(y - yo) / scale) <= 1e-9
