"""Shared helpers of the GPU tests: run one level through the C ABI with per-sample output."""
from __future__ import annotations

import numpy as np


def run_level(mlmc, level, M, N, first, prob, seed, precision, launch=None, tag=0):
    """(sums[4] from the device, Y per sample) via mlmc_level_sums_async on torch buffers."""
    import torch

    ws_bytes = mlmc.mlmc_level_workspace_bytes(level, M, N, precision, launch)
    ws = torch.zeros(ws_bytes, dtype=torch.uint8, device="cuda")
    d_sums = torch.zeros(4, dtype=torch.float64, device="cuda")
    d_y = torch.zeros(max(N, 1), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    mlmc.mlmc_level_sums_async(level, M, N, first, prob, seed, d_sums, ws, ws_bytes, precision=precision, tag=tag,
                               launch=launch, d_y=d_y, stream=stream)
    torch.cuda.synchronize()
    return d_sums.cpu().numpy(), d_y.cpu().numpy()[:N]


def oracle_problem(oracle, prob):
    return oracle.Problem(S0=prob.S0, r=prob.r, sigma=prob.sigma, T=prob.T, payoff=prob.payoff, K=prob.K,
                          Q=prob.cash, scheme=prob.scheme)


def moment_sums(y):
    y = np.asarray(y, dtype=np.float64)
    return np.array([y.sum(), (y ** 2).sum(), (y ** 3).sum(), (y ** 4).sum()])
