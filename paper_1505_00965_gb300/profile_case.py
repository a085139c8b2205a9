"""Launch one level kernel a few times on fixed arguments (for profilers and quick timing).

    python -m paper_1505_00965_gb300.profile_case --level 6 --N 1000000 --payoff asian \\
        --precision fp32 --reps 3
    python -m paper_1505_00965_gb300.profile_case --kind quintic --scheme tamed --payoff second_moment \\
        --level 6 --N 1000000

Prints the CUDA-event time per launch and the coupled path-steps per second.
"""
from __future__ import annotations

import argparse

from . import mlmc


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--level", type=int, default=6)
    ap.add_argument("--M", type=int, default=4)
    ap.add_argument("--N", type=int, default=1_000_000)
    ap.add_argument("--payoff", default="asian", choices=sorted(mlmc.PAYOFFS))
    ap.add_argument("--kind", default="gbm", choices=sorted(mlmc.MODELS))
    ap.add_argument("--scheme", default="em", choices=sorted(mlmc.SCHEMES))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--lanes", type=int, default=0, help="lanes per path (0 = automatic)")
    ap.add_argument("--threads", type=int, default=0, help="threads per block (0 = automatic)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--cv-mean", type=int, default=0, metavar="R",
                    help="time the control variate's lattice mean sample over R replicates instead "
                         "(a seeded random network on level 0)")
    args = ap.parse_args(argv)

    import torch

    if args.cv_mean:
        import time

        import numpy as np

        cv = mlmc.mlmc_cv_create(4, mlmc.Problem(payoff="asian"))
        theta = (np.random.default_rng(1).standard_normal(mlmc.MLMC_CV_PARAMS) * 0.2).astype(np.float32)
        mlmc.mlmc_cv_set_params(cv, 0, theta)
        d = torch.zeros(2, dtype=torch.float64, device="cuda")
        for rep in range(args.warmup + args.reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mlmc.mlmc_cv_mean_sums(cv, 0, args.cv_mean, 0, 1, d)
            dt = time.perf_counter() - t0
        print(f"cv mean sample: {args.cv_mean} replicates, {dt * 1e3:.3f} ms per call (host clock), "
              f"{dt / (args.cv_mean * mlmc.MLMC_CV_LATTICE_POINTS) * 1e9:.4f} ns per lattice point")
        return

    prob = mlmc.Problem(payoff=args.payoff, kind=args.kind, scheme=args.scheme)
    launch = {"lanes_per_path": args.lanes, "threads_per_block": args.threads}
    ws_bytes = mlmc.mlmc_level_workspace_bytes(args.level, args.M, args.N, args.precision, launch)
    ws = torch.zeros(ws_bytes, dtype=torch.uint8, device="cuda")
    d_sums = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def launch_once():
        mlmc.mlmc_level_sums_async(args.level, args.M, args.N, 0, prob, 1, d_sums, ws, ws_bytes,
                                   precision=args.precision, launch=launch, stream=stream)

    for _ in range(args.warmup):
        launch_once()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.reps):
        launch_once()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.reps, 1)
    steps = args.N * args.M ** args.level
    print(f"level={args.level} M={args.M} N={args.N} model={args.kind} scheme={args.scheme} payoff={args.payoff} "
          f"precision={args.precision}: "
          f"{ms:.4f} ms/launch, {steps / ms / 1e6:.4g} G coupled steps/s, sums={d_sums.tolist()}")


if __name__ == "__main__":
    main()
