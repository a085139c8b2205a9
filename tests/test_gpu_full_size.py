"""Parity at the benchmark's full sizes and at the engine's limits.

* Benchmark workload, full size: the adaptive estimates to eps = 1e-3 of the arithmetic-Asian
  and the fixed-strike lookback call (GBM S0 = K = 100, r = 0.05, sigma = 0.2, T = 1, M = 4,
  L <= 8, N0 = 1e4, FP32 paths and FP64 sums; Sec. 5's adaptive algorithm).  Each level's whole
  sample range [0, N_l) then runs as one launch in the planner's launch shape with per-sample
  output.  Sampled samples (both ends of the range, its middle and seeded random indices) are
  compared with the oracle one by one; the device's four sums are compared with the sums of its
  own samples over the whole range (a property that holds at any size); and the driver's
  per-level sums, accumulated over its rounds, with the single launch.
* Longest paths: M^l = 2^24 fine steps (M = 4, l = 12 and M = 8, l = 8), the limit of the ABI,
  and the deepest level index (M = 2, l = 15).
* Sample indices at the top of the 64-bit range: ranges whose exclusive end is 2^64 - 1, the
  largest the ABI accepts, on every kernel form (level 0 packs four samples into one Philox
  block; M = 2 level 1 packs two).

Per-sample bound as in the level parity tests: |Y_gpu - Y_oracle| <= 8 (u sqrt(n + 1) + e_z)
S0 e^{rT}, with n = M^l, u the unit roundoff of the path precision and e_z the normals' error.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import ode

from gpu_helpers import moment_sums, oracle_problem, run_level

pytestmark = pytest.mark.gpu

GBM = dict(S0=100.0, r=0.05, sigma=0.2, T=1.0, K=100.0, cash=1.0)
U = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24}
EZ = {"fp64": 1e-15, "fp32": 2e-6}
TOP = 2 ** 64


@pytest.fixture(scope="module")
def mlmc():
    from paper_1505_00965_gb300 import build

    build.build()
    from paper_1505_00965_gb300 import mlmc as binding

    return binding


def _bound(precision, level, M):
    return 8.0 * (U[precision] * math.sqrt(M ** level + 1) + EZ[precision]) * GBM["S0"] * math.exp(GBM["r"] * GBM["T"])


def _sampled_indices(N, rng, n_random=40):
    idx = set(range(min(N, 8))) | set(range(max(0, N - 8), N)) | {N // 2 - 1, N // 2}
    idx |= set(int(i) for i in rng.integers(0, N, size=n_random))
    return sorted(i for i in idx if 0 <= i < N)


def _device_moments(y, chunk=1 << 27):
    """sum y^k and sum |y|^k (k = 1..4) of a device vector, in FP64 on the device."""
    import torch

    s = torch.zeros(4, dtype=torch.float64, device=y.device)
    a = torch.zeros(4, dtype=torch.float64, device=y.device)
    for i in range(0, y.numel(), chunk):
        v = y[i:i + chunk]
        av = v.abs()
        pv, pa = v.clone(), av.clone()
        for k in range(4):
            if k:
                pv.mul_(v)
                pa.mul_(av)
            s[k] += pv.sum()
            a[k] += pa.sum()
    return s.cpu().numpy(), a.cpu().numpy()


@pytest.fixture(scope="module")
def benchmark_estimates(mlmc):
    """The benchmark's adaptive estimates (seed 1) of both payoffs."""
    out = {}
    for payoff in ("asian", "lookback"):
        p = mlmc.Problem(payoff=payoff, **GBM)
        out[payoff] = (p, mlmc.mlmc_estimate(1e-3, p, 1, M=4, Lmin=2, Lmax=8, N0=10_000))
    return out


@pytest.mark.parametrize("payoff", ["asian", "lookback"])
def test_benchmark_workload_full_size(mlmc, benchmark_estimates, payoff):
    import torch

    p, est = benchmark_estimates[payoff]
    op = oracle_problem(oracle, p)
    seed, M = 1, 4
    assert est.L >= 3 and len(est.N) == est.L + 1
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(2024)
    scale = abs(est.sums[0][0] / est.N[0])
    for level, N in enumerate(est.N):
        need = 8 * N
        free, _ = torch.cuda.mem_get_info()
        assert need < free // 2, f"level {level}: {N} samples need {need / 2**30:.1f} GiB of per-sample output"
        ws_bytes = mlmc.mlmc_level_workspace_bytes(level, M, N, "fp32")
        ws = torch.zeros(ws_bytes, dtype=torch.uint8, device="cuda")
        d_sums = torch.zeros(4, dtype=torch.float64, device="cuda")
        d_y = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        mlmc.mlmc_level_sums_async(level, M, N, 0, p, seed, d_sums, ws, ws_bytes, precision="fp32", d_y=d_y,
                                   stream=stream)
        torch.cuda.synchronize()
        sums = d_sums.cpu().numpy()
        # sampled samples against the oracle, one by one
        idx = _sampled_indices(N, rng)
        y = d_y[torch.tensor(idx, device="cuda")].cpu().numpy()
        yo = np.array([oracle.level_samples(level, M, 1, op, seed=seed, first=i, stream="fp32")[0] for i in idx])
        bound = _bound("fp32", level, M)
        assert np.all(np.isfinite(y)), level
        worst = float(np.max(np.abs(y - yo)))
        assert worst <= bound, (level, worst, bound)
        # the device's sums against the sums of its own samples over the whole range
        own, absk = _device_moments(d_y)
        for k in range(4):
            assert abs(sums[k] - own[k]) <= 32 * U["fp32"] * absk[k] + 1e-300, (level, k, sums[k], own[k])
        # the driver's rounds compose to the same samples
        m_single = sums[0] / N
        assert abs(est.sums[level][0] / N - m_single) <= 1e-5 * max(abs(m_single), scale), level
        del d_y, ws
        torch.cuda.empty_cache()


@pytest.mark.parametrize("M,level", [(4, 12), (8, 8), (2, 15)])
@pytest.mark.parametrize("payoff,precision,lanes", [("lookback", "fp32", 0), ("asian", "fp32", 0), ("lookback", "fp64", 0),
                                                    ("asian", "fp32", 1)])
def test_longest_paths(mlmc, M, level, payoff, precision, lanes):
    """M^l at the ABI's limit of 2^24 fine steps (and the deepest level index), split over lanes
    by the planner (lanes 0) or run by one thread per path: the FP32 arithmetic-Asian running
    sum then adds 2^24 values in one thread, in partials of 256 steps."""
    N, first, seed = 3, 5, 77
    p = mlmc.Problem(payoff=payoff, **GBM)
    op = oracle_problem(oracle, p)
    launch = {"lanes_per_path": lanes} if lanes else None
    sums, y = run_level(mlmc, level, M, N, first, p, seed, precision, launch=launch)
    yo = oracle.level_samples(level, M, N, op, seed=seed, first=first, stream=precision)
    assert np.all(np.isfinite(y))
    assert np.max(np.abs(y - yo)) <= _bound(precision, level, M)
    own = moment_sums(y)
    for k in range(4):
        assert abs(sums[k] - own[k]) <= 32 * U["fp32"] * np.sum(np.abs(y) ** (k + 1)) + 1e-300


def test_beyond_longest_paths_is_rejected(mlmc):
    p = mlmc.Problem(payoff="asian", **GBM)
    for M, level in [(4, 13), (8, 9), (2, 16)]:
        with pytest.raises(mlmc.MLMCError) as ei:
            mlmc.mlmc_level_sums_ex(level, M, 1, 0, p, 1)
        assert ei.value.status == mlmc.MLMC_EINVAL


TOP_RANGES = [(TOP - 2, 1), (TOP - 3, 2), (TOP - 7, 6), (TOP - 1001, 1000)]
# (name, M, level, problem fields, oracle mode); every kernel form the engine selects
TOP_CASES = [
    ("level0_lookback", 4, 0, dict(payoff="lookback"), oracle.MODE_COUPLED),
    ("level0_milstein_asian", 4, 0, dict(payoff="asian", scheme="milstein"), oracle.MODE_COUPLED),
    ("M2_level1_asian", 2, 1, dict(payoff="asian"), oracle.MODE_COUPLED),
    ("M4_level1_straight_line", 4, 1, dict(payoff="asian"), oracle.MODE_COUPLED),
    ("M4_level3_lookback", 4, 3, dict(payoff="lookback"), oracle.MODE_COUPLED),
    ("M4_level5_split8", 4, 5, dict(payoff="asian"), oracle.MODE_COUPLED),
    ("M4_level1_ns2", 4, 1, dict(payoff="asian"), oracle.MODE_COUPLED),
    ("M4_level3_lookback_ns2", 4, 3, dict(payoff="lookback"), oracle.MODE_COUPLED),
    ("antithetic_M4_level2", 4, 2, dict(payoff="asian", estimator="antithetic"), oracle.MODE_ANTITHETIC),
    ("antithetic_M2_level1", 2, 1, dict(payoff="lookback", estimator="antithetic"), oracle.MODE_ANTITHETIC),
]


@pytest.mark.parametrize("first,N", TOP_RANGES)
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name,M,level,fields,mode", TOP_CASES, ids=[c[0] for c in TOP_CASES])
def test_sample_indices_at_top_of_64_bits(mlmc, name, M, level, fields, mode, precision, first, N):
    """Samples are addressed by 64-bit index (the stream's counter words s_lo, s_hi): ranges
    up to the largest accepted end, 2^64 - 1, give the oracle's samples, including partly
    covered Philox blocks."""
    seed = 31
    p = mlmc.Problem(**fields, **GBM)
    op = oracle_problem(oracle, p)
    launch = {"lanes_per_path": 8} if name.endswith("split8") else None
    if name.endswith("ns2"):
        if precision != "fp32":
            pytest.skip("two samples per thread: FP32 kernels")
        launch = {"lanes_per_path": 1, "samples_per_thread": 2}
    sums, y = run_level(mlmc, level, M, N, first, p, seed, precision, launch=launch)
    yo = oracle.level_samples(level, M, N, op, seed=seed, first=first, stream=precision, mode=mode)
    assert np.all(np.isfinite(y))
    assert np.max(np.abs(y - yo)) <= _bound(precision, level, M)
    own = moment_sums(y)
    red_tol = 1e-12 if precision == "fp64" else 32 * U["fp32"]
    for k in range(4):
        assert abs(sums[k] - own[k]) <= red_tol * np.sum(np.abs(y) ** (k + 1)) + 1e-300


@pytest.mark.parametrize("first,N", TOP_RANGES)
@pytest.mark.parametrize("level", [0, 2])
def test_quintic_sample_indices_at_top_of_64_bits(mlmc, level, first, N):
    """The quintic ODE kernel packs four samples per Philox block at every level."""
    seed = 31
    p = mlmc.Problem(kind="quintic", scheme="tamed", payoff="second_moment", T=1.0)
    _, y = run_level(mlmc, level, 4, N, first, p, seed, "fp64")
    yo = ode.level_samples(level, 4, N, 1.0, seed, "tamed", first=first, stream="fp64")
    x0 = ode.initial_values(level, first, N, seed, stream="fp64")
    n = 4 ** level
    tol = 8.0 * (1.0 + x0 ** 2) * (EZ["fp64"] + 4 * U["fp64"] * math.sqrt(n + 1))
    assert np.all(np.abs(y - yo) <= tol)


@pytest.mark.parametrize("estimator,mode", [("coupled", oracle.MODE_COUPLED), ("antithetic", oracle.MODE_ANTITHETIC)])
@pytest.mark.parametrize("scheme", ["em", "milstein"])
@pytest.mark.parametrize("M,level,lanes", [(4, 7, 1), (2, 13, 1), (4, 8, 2), (2, 14, 4), (4, 7, -2), (2, 13, -2)])
def test_long_lane_kernels(mlmc, M, level, lanes, scheme, estimator, mode):
    """Lanes of more than 4096 steps take the FP32 arithmetic-Asian kernels that add the running
    sum in partials of 256 steps (one thread per path, and split paths; lanes = -2: one thread
    per path, two samples per thread)."""
    if estimator == "antithetic" and lanes != 1:
        pytest.skip("the antithetic estimator runs one thread per path, one sample per thread")
    if lanes == -2 and scheme != "em":
        pytest.skip("two samples per thread: Euler--Maruyama kernels")
    N, first, seed = 67, 2 ** 40 + 1, 5
    p = mlmc.Problem(payoff="asian", scheme=scheme, estimator=estimator, **GBM)
    op = oracle_problem(oracle, p)
    launch = ({"lanes_per_path": lanes} if lanes > 1 else
              {"lanes_per_path": 1, "samples_per_thread": 2} if lanes == -2 else {"lanes_per_path": 1})
    sums, y = run_level(mlmc, level, M, N, first, p, seed, "fp32", launch=launch)
    yo = oracle.level_samples(level, M, N, op, seed=seed, first=first, stream="fp32", mode=mode)
    assert np.max(np.abs(y - yo)) <= _bound("fp32", level, M)
    own = moment_sums(y)
    for k in range(4):
        assert abs(sums[k] - own[k]) <= 32 * U["fp32"] * np.sum(np.abs(y) ** (k + 1)) + 1e-300
