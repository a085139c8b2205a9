"""The autotuner on the GPU: it fills the table, and the shapes it picks keep every sample equal
to the oracle's within the level tolerances (launch shapes never change the samples)."""
import numpy as np
import pytest

import oracle

from gpu_helpers import oracle_problem, run_level

pytestmark = pytest.mark.gpu

GBM = dict(S0=100.0, r=0.05, sigma=0.2, T=1.0, K=100.0, cash=1.0)


@pytest.fixture()
def mlmc():
    from paper_1505_00965_gb300 import build

    build.build()
    from paper_1505_00965_gb300 import mlmc as binding

    binding.mlmc_autotune_clear()
    yield binding
    binding.mlmc_autotune_clear()


def test_autotune_then_parity(mlmc, tmp_path):
    n = mlmc.mlmc_autotune(M=4, max_level=5, precision="fp32", payoff="asian")
    assert n > 0 and mlmc.mlmc_autotune_entries() == n
    for level in range(6):
        shape = mlmc.mlmc_autotune_lookup("fp32", "asian", 4, level, 1 << 16)
        assert shape is not None and shape[0] in (128, 256, 512) and shape[1] in (1, 2, 4, 8, 16, 32)
        assert shape[3] in (1, 2) and (shape[3] == 1 or (shape[1] == 1 and level >= 1 and shape[0] <= 512))
    p = mlmc.Problem(payoff="asian", **GBM)
    op = oracle_problem(oracle, p)
    for level, N in [(0, 5000), (3, 2000), (5, 600)]:
        sums, y = run_level(mlmc, level, 4, N, 9, p, 3, "fp32")
        yo = oracle.level_samples(level, 4, N, op, seed=3, first=9, stream="fp32")
        bound = 8.0 * (2.0 ** -24 * np.sqrt(4 ** level + 1) + 2e-6) * 100.0 * np.exp(0.05)
        assert np.max(np.abs(y - yo)) <= bound
    path = tmp_path / "t.json"
    mlmc.mlmc_autotune_save(str(path))
    mlmc.mlmc_autotune_clear()
    assert mlmc.mlmc_autotune_load(str(path)) == n
    est = mlmc.mlmc_estimate(1e-2, p, 1)
    assert est.converged


def test_tuned_two_samples_per_thread_keeps_parity(mlmc, tmp_path):
    """A table entry with two samples per thread (as the tuner may choose for FP32 whole paths)
    drives the planner's launches, which keep every sample equal to the oracle's; on levels where
    the two-sample kernel does not exist (level 0) the planner falls back to one sample."""
    path = tmp_path / "ns2.json"
    lines = []
    for level in (0, 1, 3, 5):
        lines.append(f' {{"precision": 1, "payoff": 2, "M": 4, "level": {level}, "log2N": 10, "threads": 128, '
                     f'"lanes": 1, "oversub": 2, "ns_per_sample": 1.0, "samples_per_thread": 2}}')
    path.write_text('{"entries": [\n' + ",\n".join(lines) + "\n]}\n")
    assert mlmc.mlmc_autotune_load(str(path)) == 4
    assert mlmc.mlmc_autotune_lookup("fp32", "lookback", 4, 3, 5000) == (128, 1, 2, 2)
    p = mlmc.Problem(payoff="lookback", **GBM)
    op = oracle_problem(oracle, p)
    for level, N in [(0, 5003), (1, 4001), (3, 2001), (5, 601)]:
        sums, y = run_level(mlmc, level, 4, N, 13, p, 3, "fp32")
        yo = oracle.level_samples(level, 4, N, op, seed=3, first=13, stream="fp32")
        bound = 8.0 * (2.0 ** -24 * np.sqrt(4 ** level + 1) + 2e-6) * 100.0 * np.exp(0.05)
        assert np.max(np.abs(y - yo)) <= bound, level
        assert abs(sums[0] - y.sum()) <= 32 * 2.0 ** -24 * np.abs(y).sum()
    est = mlmc.mlmc_estimate(1e-2, p, 2)
    assert est.L >= 2
