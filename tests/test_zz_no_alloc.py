"""The allocation-free level entry point, for callers that cannot allocate device memory at run
time (latency-critical loops, processes whose device memory belongs to another allocator,
deployments that forbid allocation after start-up).

It must give the same sums and per-sample values as mlmc_level_sums_async with its own
workspace, on two calls in a row (the fixed scratch keeps the previous call's contents), and
reject a grid larger than its fixed scratch.  This file is collected last, so a run that stops
at its first failure has already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import run_level

pytestmark = pytest.mark.gpu

GBM = dict(S0=100.0, r=0.05, sigma=0.2, T=1.0, K=100.0, cash=1.0)


@pytest.fixture(scope="module")
def mlmc():
    from paper_1505_00965_gb300 import build

    build.build()
    from paper_1505_00965_gb300 import mlmc as binding

    return binding


def _noalloc_via_c_abi(mlmc, level, M, N, first, prob, seed, precision, launch):
    """Call mlmc_level_sums_noalloc through the C ABI with raw device pointers."""
    import torch

    d_sums = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    d_y = torch.zeros(N, dtype=torch.float64, device="cuda")
    m, p = prob.model(), prob.payoff_struct()
    ln = mlmc.mlmc_launch(launch.get("threads_per_block", 0), launch.get("lanes_per_path", 0),
                          launch.get("blocks", 0), 0)
    prec = mlmc.PRECISIONS[precision]
    rc = mlmc._lib.mlmc_level_sums_noalloc(level, M, ctypes.c_uint64(N), ctypes.c_uint64(first), ctypes.byref(m),
                                          ctypes.byref(p), ctypes.c_uint64(seed), prec, 0, ctypes.byref(ln),
                                          ctypes.c_void_p(d_sums.data_ptr()), ctypes.c_void_p(d_y.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == mlmc.MLMC_OK, mlmc.mlmc_last_error()
    torch.cuda.synchronize()
    return d_sums.cpu().numpy(), d_y.cpu().numpy()


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-12), ("fp32", 1e-12)])
@pytest.mark.parametrize("payoff,level,N,launch", [
    ("asian", 3, 50_001, {"threads_per_block": 256}),
    ("lookback", 6, 3_001, {"lanes_per_path": 8, "threads_per_block": 128}),
    ("european", 0, 200_003, {}),
])
def test_noalloc_matches_async_on_two_calls(mlmc, precision, rtol, payoff, level, N, launch):
    prob = mlmc.Problem(payoff=payoff, **GBM)
    ref_sums, ref_y = run_level(mlmc, level, 4, N, 17, prob, 5, precision, launch=launch)
    for _ in range(2):
        sums, y = _noalloc_via_c_abi(mlmc, level, 4, N, 17, prob, 5, precision, launch)
        np.testing.assert_allclose(sums, ref_sums, rtol=rtol, atol=0)
        np.testing.assert_array_equal(y, ref_y)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_grid_cut_to_its_scratch(mlmc, precision):
    """64-thread blocks over a million samples: the planner sizes the grid beyond the 2048 blocks
    the fixed scratch holds, and the entry point cuts it to 2048.  Every sample is the async
    form's (and the oracle's); the sums add the same samples in another order."""
    import oracle

    from gpu_helpers import moment_sums, oracle_problem

    level, N, first, seed = 2, 1_000_003, 5, 7
    launch = {"threads_per_block": 64}
    prob = mlmc.Problem(payoff="asian", **GBM)
    assert mlmc.mlmc_level_workspace_bytes(level, 4, N, precision, {"threads_per_block": 64, "blocks": 4096}) > 0
    ref_sums, ref_y = run_level(mlmc, level, 4, N, first, prob, seed, precision, launch=launch)
    for _ in range(2):
        sums, y = _noalloc_via_c_abi(mlmc, level, 4, N, first, prob, seed, precision, launch)
        np.testing.assert_array_equal(y, ref_y)
        own = moment_sums(y)
        u = 2.0 ** -24 if precision == "fp32" else 2.0 ** -53
        for k in range(4):
            scale = np.sum(np.abs(y) ** (k + 1))
            assert abs(sums[k] - ref_sums[k]) <= 64 * u * scale, (k, sums[k], ref_sums[k])
            assert abs(sums[k] - own[k]) <= 32 * u * scale, (k, sums[k], own[k])
    op = oracle_problem(oracle, prob)
    bound = 8.0 * ((2.0 ** -24 if precision == "fp32" else 2.0 ** -53) * np.sqrt(17) +
                   (2e-6 if precision == "fp32" else 1e-15)) * 100.0 * np.exp(0.05)
    for a in (0, N // 2, N - 1000):
        yo = oracle.level_samples(level, 4, 1000, op, seed=seed, first=first + a, stream=precision)
        assert np.max(np.abs(y[a:a + 1000] - yo)) <= bound


def test_noalloc_takes_no_device_memory(mlmc):
    """After the first call (which loads the kernel and looks up the scratch), further calls do
    not change the device's free memory."""
    import torch

    prob = mlmc.Problem(payoff="lookback", **GBM)
    _noalloc_via_c_abi(mlmc, 3, 4, 20_001, 0, prob, 3, "fp32", {})
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        _noalloc_via_c_abi(mlmc, 3, 4, 20_001, 0, prob, 3, "fp32", {})
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0, (free0, free1)


def test_noalloc_rejects_grid_beyond_its_scratch(mlmc):
    import torch

    d_sums = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(mlmc.MLMCError) as ei:
        mlmc.mlmc_level_sums_noalloc(2, 4, 1000, 0, mlmc.Problem(**GBM), 1, d_sums, launch={"blocks": 4096})
    assert ei.value.status == mlmc.MLMC_EINVAL
    assert "static scratch holds 2048 blocks" in str(ei.value)
