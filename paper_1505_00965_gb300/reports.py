"""Reference workloads beyond the benchmark step, as JSON reports.

    python -m paper_1505_00965_gb300.reports precision [--samples 10000000]
    python -m paper_1505_00965_gb300.reports sec6
    python -m paper_1505_00965_gb300.reports milstein

precision  FP32 against FP64 path arithmetic on the identical random stream (the FP32 path's
           samples computed both ways): digital call (cash 1) and arithmetic-Asian call, levels
           0..7 of M = 4, per-level mean and variance and their FP32 errors.
sec6       the experiment of Sec. 6: GBM dX = 0.05 X dt + 0.25 X dW, X(0) = 100, T = 1, European
           call and digital call (cash 100), eps = 0.1, 0.05, 0.02, 0.01, 0.005; per eps the
           MLMC N_l, eps^2 * cost, and the eps^2 * cost of standard Monte Carlo at the same finest
           step (N = 2 eps^-2 Var(P_L), cost N M^L).
milstein   time-to-eps and eps^2 * cost of Euler--Maruyama and Milstein MLMC (European call).
antithetic the antithetic estimator of Sec. 7 against the coupled one: per level Var Y_l (2^20
           samples; Asian and lookback calls, Euler--Maruyama and Milstein), and adaptive
           estimates (eps^2 * cost, time-to-eps) at eps = 1e-3 and 5e-4.
tamed      the counterexample of Sec. 5 (Eq. count), dX = -X^5 dt, X(0) ~ N(0, 1), E[X(1)^2]:
           per level and scheme (explicit / tamed Euler--Maruyama) the mean, variance and number
           of non-finite samples of Y_l over 2^20 samples, FP32 and FP64; the adaptive estimates
           with each scheme against the exact value (quadrature of E[X0^2 (1 + 4 X0^4)^(-1/2)]).
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import mlmc

GBM = dict(S0=100.0, r=0.05, sigma=0.2, T=1.0, K=100.0)


def _level_moments(level, M, N, prob, seed, precision):
    sums, _ = mlmc.mlmc_level_sums_ex(level, M, N, 0, prob, seed, precision=precision)
    m = sums[0] / N
    return m, max(sums[1] / N - m * m, 0.0)


def precision_sweep(samples: int = 10_000_000, levels=range(8), M: int = 4, seed: int = 1) -> dict:
    out = {"samples_per_level": samples, "M": M, "payoffs": {}}
    for payoff in ("digital", "asian"):
        prob = mlmc.Problem(payoff=payoff, cash=1.0, **GBM)
        rows = []
        for level in levels:
            n = samples if level < 6 else max(samples // 4 ** (level - 5), 100_000)
            m32, v32 = _level_moments(level, M, n, prob, seed, "fp32")
            m64, v64 = _level_moments(level, M, n, prob, seed, "fp64_stream32")
            rows.append({"level": level, "samples": n, "mean_fp64": m64, "var_fp64": v64,
                         "mean_err_fp32": m32 - m64, "var_rel_err_fp32": (v32 - v64) / v64 if v64 else None,
                         "mean_std_error": math.sqrt(v64 / n)})
        out["payoffs"][payoff] = rows
    return out


def sec6(seed: int = 1, M: int = 4) -> dict:
    out = {"model": "dX = 0.05 X dt + 0.25 X dW, X(0) = 100, T = 1, K = 100", "M": M, "options": {}}
    for payoff, cash in (("european", 1.0), ("digital", 100.0)):
        prob = mlmc.Problem(payoff=payoff, S0=100.0, r=0.05, sigma=0.25, T=1.0, K=100.0, cash=cash)
        single = mlmc.Problem(payoff=payoff, S0=100.0, r=0.05, sigma=0.25, T=1.0, K=100.0, cash=cash,
                              estimator="single")
        rows = []
        for eps in (0.1, 0.05, 0.02, 0.01, 0.005):
            est = mlmc.mlmc_estimate(eps, prob, seed, M=M, Lmin=2, Lmax=10, N0=10_000)
            L = est.L
            _, vL = _level_moments(L, M, 200_000, single, seed + 1000, "fp32")
            n_std = math.ceil(2.0 / eps ** 2 * vL)
            rows.append({"eps": eps, "P": est.P, "L": L, "N": est.N, "eps2_cost_mlmc": eps ** 2 * est.total_cost,
                         "eps2_cost_std_mc": eps ** 2 * n_std * M ** L, "time_ms_mlmc": est.wall_ms,
                         "converged": est.converged})
        out["options"][payoff] = rows
    return out


def milstein(seed: int = 1, M: int = 4) -> dict:
    rows = []
    for scheme in ("em", "milstein"):
        prob = mlmc.Problem(payoff="european", scheme=scheme, **GBM)
        for eps in (1e-2, 1e-3, 5e-4):
            est = mlmc.mlmc_estimate(eps, prob, seed, M=M)
            rows.append({"scheme": scheme, "eps": eps, "P": est.P, "L": est.L, "beta": est.beta,
                         "eps2_cost": eps ** 2 * est.total_cost, "time_to_eps_ms": est.wall_ms})
    return {"payoff": "european", "rows": rows}


def quintic_exact(T: float = 1.0) -> float:
    """E[X(T)^2] for dX = -X^5 dt, X(0) ~ N(0, 1): X(T) = X0 (1 + 4 T X0^4)^(-1/4)."""
    from scipy import integrate

    f = lambda x: x * x / math.sqrt(1.0 + 4.0 * T * x ** 4) * math.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return integrate.quad(f, -math.inf, math.inf, epsabs=1e-14, epsrel=1e-12)[0]


def tamed(seed: int = 1, M: int = 4, samples: int = 1 << 20) -> dict:
    import torch

    out = {"model": "dX = -X^5 dt, X(0) ~ N(0,1), T = 1, quantity E[X(T)^2]", "exact": quintic_exact(1.0),
           "samples_per_level": samples, "levels": [], "estimates": []}
    d_y = torch.zeros(samples, dtype=torch.float64, device="cuda")
    d_s = torch.zeros(4, dtype=torch.float64, device="cuda")
    for precision in ("fp32", "fp64"):
        for scheme in ("em", "tamed"):
            prob = mlmc.Problem(kind="quintic", scheme=scheme, payoff="second_moment", T=1.0)
            for level in range(0, 8):
                wsb = mlmc.mlmc_level_workspace_bytes(level, M, samples, precision)
                ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
                mlmc.mlmc_level_sums_async(level, M, samples, 0, prob, seed, d_s, ws, wsb, precision=precision,
                                           d_y=d_y)
                torch.cuda.synchronize()
                y = d_y.cpu().numpy()
                bad = int((~np.isfinite(y)).sum())
                fin = y[np.isfinite(y)]
                out["levels"].append({"precision": precision, "scheme": scheme, "level": level, "non_finite": bad,
                                      "mean": float(fin.mean()), "var": float(fin.var()),
                                      "max_abs": float(np.abs(fin).max())})
    for precision in ("fp32", "fp64"):
        for scheme in ("em", "tamed"):
            prob = mlmc.Problem(kind="quintic", scheme=scheme, payoff="second_moment", T=1.0)
            for eps in (1e-2, 3e-3, 1e-3):
                try:
                    est = mlmc.mlmc_estimate(eps, prob, seed, M=M, precision=precision)
                    out["estimates"].append({"precision": precision, "scheme": scheme, "eps": eps, "P": est.P,
                                             "error": est.P - out["exact"], "L": est.L, "N": est.N,
                                             "alpha": est.alpha, "beta": est.beta, "time_to_eps_ms": est.wall_ms,
                                             "converged": est.converged})
                except mlmc.MLMCError as e:
                    out["estimates"].append({"precision": precision, "scheme": scheme, "eps": eps,
                                             "status": e.status, "error_message": str(e)})
    return out


def antithetic(seed: int = 1, M: int = 4, samples: int = 1 << 20) -> dict:
    out = {"model": "GBM S0 = K = 100, r = 0.05, sigma = 0.2, T = 1", "M": M, "samples_per_level": samples,
           "levels": [], "estimates": []}
    for payoff in ("asian", "lookback"):
        for scheme in ("em", "milstein"):
            for level in range(1, 8):
                n = samples if level < 6 else samples // 4
                row = {"payoff": payoff, "scheme": scheme, "level": level, "samples": n}
                for est in ("coupled", "antithetic"):
                    prob = mlmc.Problem(payoff=payoff, scheme=scheme, estimator=est, **GBM)
                    m, v = _level_moments(level, M, n, prob, seed, "fp32")
                    row[f"var_{est}"] = v
                    row[f"mean_{est}"] = m
                out["levels"].append(row)
    for payoff, scheme in (("asian", "milstein"), ("asian", "em"), ("lookback", "em")):
        for eps in (1e-3, 5e-4):
            for est in ("coupled", "antithetic"):
                prob = mlmc.Problem(payoff=payoff, scheme=scheme, estimator=est, **GBM)
                mlmc.mlmc_estimate(eps, prob, seed, M=M)  # warm
                e = mlmc.mlmc_estimate(eps, prob, seed, M=M)
                out["estimates"].append({"payoff": payoff, "scheme": scheme, "estimator": est, "eps": eps, "P": e.P,
                                         "L": e.L, "beta": e.beta, "eps2_cost": eps ** 2 * e.total_cost,
                                         "time_to_eps_ms": e.wall_ms, "converged": e.converged})
    return out


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("report", choices=["precision", "sec6", "milstein", "tamed", "antithetic"])
    ap.add_argument("--samples", type=int, default=10_000_000)
    args = ap.parse_args(argv)
    if args.report == "precision":
        res = precision_sweep(args.samples)
    elif args.report == "sec6":
        res = sec6()
    elif args.report == "milstein":
        res = milstein()
    elif args.report == "antithetic":
        res = antithetic()
    else:
        res = tamed()
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
