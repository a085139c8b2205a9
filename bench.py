#!/usr/bin/env python3
"""Benchmark: adaptive multilevel Monte Carlo on GB300, one JSON line on rank 0.

Workload (one step): adaptive MLMC estimates to root-mean-square accuracy eps = 1e-3 of the
arithmetic-Asian call and the fixed-strike lookback call on GBM (S0 = K = 100, r = 0.05,
sigma = 0.2, T = 1), M = 4, levels up to 8, 10^4 warm-up samples per level, FP32 paths with
FP64 moment sums, seeds 1..8 (rank r takes seeds 8r+1..8r+8: per-GPU work is fixed).

  value  coupled path-steps/s of the whole step (sum over estimates of sum_l N_l M^l), timed
         with CUDA events on the stream the engine runs on
  e2e    the same metric through the public C ABI (mlmc_estimate: host arguments, host result,
         the per-round device-to-host copies inside) timed by the host clock

`--impl reference` times the FP64 CPU oracle instead (a bounded sample of the workload on the
host cores).  Under torchrun only rank 0 runs that arm.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import select
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLMC time-to-ε (ε=1e-3) & coupled path-steps/s vs plain FP64 GPU MLMC"
UNIT = "coupled path-steps/s"
GBM = dict(S0=100.0, r=0.05, sigma=0.2, T=1.0, K=100.0)
PAYOFFS = ("asian", "lookback")
M, LMIN, LMAX, N0, EPS = 4, 2, 8, 10_000, 1e-3
SEEDS_PER_RANK = 8
WORKLOAD = ("adaptive MLMC to eps=1e-3: arithmetic-Asian and fixed-strike lookback calls, GBM S0=K=100 "
            "r=0.05 sigma=0.2 T=1, M=4, L<=8, N0=1e4, FP32 paths + FP64 sums, seeds 1..8 per GPU")
# GB300 issue limit: 4 schedulers per SM, each issuing one warp instruction (32 lanes) per clock.
SCHEDULERS_PER_SM, WARP = 4, 32
SM_MAX_MHZ_FALLBACK = 2070.0


# ------------------------------------------------------------------ helpers (CPU-testable)

def rank_seeds(rank: int, n: int = SEEDS_PER_RANK) -> list[int]:
    """Seeds of one rank: ranks draw disjoint seeds, so the estimates are independent."""
    return [rank * n + i + 1 for i in range(n)]


def level_instructions(level: int, m: int, payoff: str) -> float:
    """Algorithmic instructions of one FP32 sample on level l, with n = M^l fine steps:
    Philox4x32-10 = 40 per block of 4 normals (10 rounds of 2 widening multiplies + 2
    three-input xors) and n / 4 blocks per sample (on levels with n < 4, 4 / n samples share a
    block); Box--Muller = 11 per pair of normals (2 mantissa builds, 2 subtractions, 3
    multiplies, 4 MUFU), n / 2 pairs; per fine step 2 (increment, step) + 1 (coarse sum, l > 0);
    per coarse step 1; running payoff functional 1 per fine and per coarse step (Asian,
    lookback); per sample 11 (payoffs, difference, moment updates)."""
    nf = m ** level
    functional = 1 if payoff in ("asian", "lookback") else 0
    per_fine = 2 + (1 if level > 0 else 0) + functional
    coarse = (nf // m) * (1 + functional) if level > 0 else 0
    return 40.0 * nf / 4 + 11.0 * nf / 2 + per_fine * nf + coarse + 11.0


def estimate_instructions(N: list[int], m: int, payoff: str) -> float:
    return sum(n * level_instructions(l, m, payoff) for l, n in enumerate(N))


def parse_clock_lines(lines: list[str]) -> dict:
    """Median SM clock, max clock and the throttle reasons seen, from nvidia-smi CSV lines of
    index, clocks.sm, clocks.max.sm, power.draw, active, hw_slowdown, hw_thermal, sw_thermal,
    sw_power_cap."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for name, val in zip(names, f[5:9]):
            if val.lower().startswith("active"):
                reasons.add(name)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def bias_estimate(mean: list, alpha: float, m: int = M) -> float:
    """The driver's bias estimate on the finest two levels, max(|m_L|, |m_{L-1}| / M^alpha) /
    (M^alpha - 1) (Theorem of Sec. 5: the estimate's bias is what MSE < eps^2 leaves to it)."""
    ma = m ** max(alpha, 0.5)
    return max(abs(mean[-1]), abs(mean[-2]) / ma) / (ma - 1.0)


def combine_over_ranks(dev_s: float, wall_s: float, steps: float, launches: float, group=None) -> tuple:
    """Max of the times and sum of the work over ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist

    if group is None and not (dist.is_available() and dist.is_initialized()):
        return dev_s, wall_s, steps, launches
    t = torch.tensor([dev_s, wall_s], dtype=torch.float64)
    w = torch.tensor([steps, launches], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t, w = t.cuda(), w.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(w, op=dist.ReduceOp.SUM, group=group)
    return float(t[0]), float(t[1]), float(w[0]), float(w[1])


# ------------------------------------------------------------------ CPU oracle arm

def _oracle_job(args):
    payoff, seed, eps = args
    sys.path.insert(0, ROOT)
    from oracle import Problem, driver

    t = time.perf_counter()
    e = driver.estimate(eps, Problem(payoff=payoff, Q=1.0, **GBM), seed, M=M, Lmin=LMIN, Lmax=LMAX, N0=N0,
                        stream="fp32")
    dt = time.perf_counter() - t
    return sum(n * M ** l for l, n in enumerate(e.N)), dt


# DRAM bytes (read + write) of one launch of the dominant kernel, from ncu (level_ns2_kernel, lookback,
# level 6, N = 10^6, two samples per thread): the kernels read no input arrays; the algorithmic
# bytes are the block partials and the four sums (608 x 32 + 32 = 19.5 KB).
TRAFFIC_BYTES_PER_LAUNCH = 97280
TRAFFIC_BASIS = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one level_ns2_kernel launch (lookback, "
                 "level 6, N=1e6, 608 blocks); algorithmic bytes 19.5 KB of block partials")
# FP64 instructions (DFMA + DADD + DMUL, thread level) per coupled step of the FP64 Asian kernel, from
# ncu's per-opcode counters on one launch (level 6, N = 1e5, one thread per sample).
FP64_INSTR_PER_STEP = 36.51
FP64_INSTR_BASIS = ("ncu smsp__sass_thread_inst_executed_op_{dfma,dadd,dmul}_pred_on of one level_kernel<double> "
                    "launch (Asian, level 6, N=1e5): 20.76 + 8.26 + 7.50 per coupled step; deeper and shallower "
                    "levels differ by their per-sample share")

ORACLE_SAMPLE = dict(eps=2e-2, seeds=tuple(range(1, 9)))
ORACLE_SAMPLE_TEXT = ("oracle adaptive MLMC of the same two options and model at eps=2e-2 (not 1e-3), "
                      "seeds 1..8 (16 estimates), FP32 stream; estimates run in parallel processes, one per "
                      "host core")


def run_oracle_sample(pool_size: int) -> tuple[float, float, int, float]:
    """(path-steps, wall seconds, processes, summed per-process seconds) of the bounded oracle
    sample."""
    import multiprocessing as mp

    jobs = [(p, s, ORACLE_SAMPLE["eps"]) for p in PAYOFFS for s in ORACLE_SAMPLE["seeds"]]
    procs = max(1, min(pool_size, len(jobs)))
    ctx = mp.get_context("spawn")
    t = time.perf_counter()
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_job, jobs)
    wall = time.perf_counter() - t
    return float(sum(r[0] for r in res)), wall, procs, float(sum(r[1] for r in res))


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    import platform

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def cpu_baseline(pool_size: int) -> dict:
    steps, wall, procs, busy = run_oracle_sample(pool_size)
    return {"value": steps / wall, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": ORACLE_SAMPLE_TEXT,
            "wall_s": round(wall, 3), "single_thread_value": steps / busy, "cpu_model": cpu_model(),
            "host_cpus": os.cpu_count()}


def reference_arm(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    pool = os.cpu_count() or 1
    for _ in range(args.warmup):
        run_oracle_sample(pool)
    tot_steps, tot_wall, tot_busy, procs = 0.0, 0.0, 0.0, 1
    for _ in range(args.steps):
        s, w, procs, b = run_oracle_sample(pool)
        tot_steps += s
        tot_wall += w
        tot_busy += b
    value = tot_steps / tot_wall
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "reference_sample": ORACLE_SAMPLE_TEXT},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": ORACLE_SAMPLE_TEXT, "single_thread_value": tot_steps / tot_busy,
                             "cpu_model": cpu_model(), "host_cpus": os.cpu_count()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid: str | None):
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "200"]
        if device_uuid:
            cmd += ["-i", device_uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        # wait (at most 10 s) for the first sample, taken before the timed region and dropped, so
        # that nvidia-smi's start-up (process and NVML initialisation) does not overlap the first
        # timed step
        if self.proc is not None and self.proc.stdout is not None:
            ready, _, _ = select.select([self.proc.stdout], [], [], 10.0)
            if ready:
                self.proc.stdout.readline()

    def stop(self) -> dict:
        if self.proc is None:
            return parse_clock_lines([])
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return parse_clock_lines(out.splitlines())


def side_workloads(mlmc, stream) -> dict:
    """Reports outside the timed region: the 512-problem batch and the learned control variate
    (Asian call, levels 0..3 trained on 10^6 samples each, applied at eps = 5e-4)."""
    from paper_1505_00965_gb300 import workloads

    out = {}
    qs = workloads.batch_problems(512)
    t = time.perf_counter()
    res = mlmc.mlmc_estimate_batch(qs, M=M, Lmin=LMIN, Lmax=LMAX, N0=N0, stream=stream)
    wall = time.perf_counter() - t
    steps = sum(r.path_steps for r in res)
    out["batch_512"] = {"wall_ms": 1e3 * wall, "kernel_ms": res[0].kernel_ms, "rounds": res[0].rounds,
                        "path_steps": steps, "path_steps_per_s": steps / wall,
                        "converged": sum(r.converged for r in res), "problems": len(res),
                        "workload": "K~U[80,120], sigma~U[0.1,0.5], T~U[0.25,2], r=0.05, payoff uniform over "
                                    "European/Asian/lookback/digital, eps log-uniform in [1e-3,1e-2], seeds 1..512"}
    # the antithetic estimator (Sec. 7) on the benchmark's options and eps, Euler--Maruyama
    anti = {}
    for p in PAYOFFS:
        prob = mlmc.Problem(payoff=p, cash=1.0, estimator="antithetic", **GBM)
        mlmc.mlmc_estimate(EPS, prob, 1, M=M, Lmin=LMIN, Lmax=LMAX, N0=N0, stream=stream)
        times = [mlmc.mlmc_estimate(EPS, prob, s, M=M, Lmin=LMIN, Lmax=LMAX, N0=N0, stream=stream).wall_ms
                 for s in range(1, 9)]
        anti[p] = statistics.median(times)
    out["antithetic_time_to_eps_ms"] = anti
    # the same estimates with their rounds on the device (one graph launch each: a driver kernel
    # configures the level kernels by device-side graph updates) against the host rounds
    prev = mlmc.mlmc_set_driver_mode("device")
    try:
        dev = {}
        for p in PAYOFFS:
            prob = mlmc.Problem(payoff=p, cash=1.0, **GBM)
            mlmc.mlmc_estimate(EPS, prob, 1, M=M, Lmin=LMIN, Lmax=LMAX, N0=N0, stream=stream)  # builds the graph
            dev[p] = statistics.median(
                mlmc.mlmc_estimate(EPS, prob, s, M=M, Lmin=LMIN, Lmax=LMAX, N0=N0, stream=stream).wall_ms
                for s in range(1, 9))
        out["device_rounds_wall_ms"] = dev
    finally:
        mlmc.mlmc_set_driver_mode(prev)
    prob = mlmc.Problem(payoff="asian", cash=1.0, **GBM)
    # trained twice: the first call also loads the control-variate kernels (lazy module loading);
    # the second is the cost of training a further problem in a running process
    t = time.perf_counter()
    cv = mlmc.mlmc_cv_train(M, prob, seed=2024, levels=4, epochs=20, n_train=1_000_000, stream=stream)
    train_s_first = time.perf_counter() - t
    mlmc.mlmc_cv_free(cv)
    t = time.perf_counter()
    cv = mlmc.mlmc_cv_train(M, prob, seed=2024, levels=4, epochs=20, n_train=1_000_000, stream=stream)
    train_s = time.perf_counter() - t
    train_info = mlmc.mlmc_cv_train_info(cv)
    levels = []
    for l in range(4):
        i = mlmc.mlmc_cv_info(cv, l)
        levels.append({"level": l, "var_ratio": i["var_resid"] / i["var_plain"], "var_plain": i["var_plain"],
                       "var_resid": i["var_resid"], "var_g": i["var_g"], "var_lattice": i["var_lattice"],
                       "lattice_gain": i["var_g"] / i["var_lattice"] if i["var_lattice"] > 0 else None,
                       "kappa": i["kappa"], "work_ratio": i["work_ratio"],
                       "used": bool(i["used"]), "ns_per_sample_plain": 1e9 * i["t_plain"],
                       "ns_per_sample_cv": 1e9 * i["t_cv"], "ns_per_lattice_point": 1e9 * i["t_mean"]})
    eps_cv = 5e-4
    seeds = range(1, 9)
    mlmc.mlmc_estimate_cv(eps_cv, cv, 1, Lmin=LMIN, Lmax=LMAX, N0=N0, stream=stream)  # warm-up
    a = [mlmc.mlmc_estimate_cv(eps_cv, cv, s, Lmin=LMIN, Lmax=LMAX, N0=N0, stream=stream) for s in seeds]
    b = [mlmc.mlmc_estimate(eps_cv, prob, s, M=M, Lmin=LMIN, Lmax=LMAX, N0=N0, stream=stream) for s in seeds]
    c = [mlmc.mlmc_estimate(eps_cv, prob, s, M=M, Lmin=LMIN, Lmax=LMAX, N0=N0, precision="fp64", stream=stream)
         for s in seeds]
    med = lambda rs: statistics.median(r.wall_ms for r in rs)
    cv_ms, plain_ms, fp64_ms = med(a), med(b), med(c)
    saving = plain_ms - cv_ms
    out["learned_cv"] = {
        "payoff": "asian", "train_s": train_s, "train_s_first_call": train_s_first,
        "training": {k: train_info[k] for k in ("data_ms", "train_ms", "train_kernel_ms", "eval_ms", "cost_ms",
                                                "total_ms", "steps", "cluster", "levels")},
        "levels": levels, "eps": eps_cv, "seeds": "1..8 (medians)",
        "time_to_eps_ms": {"fp32_cv": cv_ms, "fp32_plain": plain_ms, "fp64_plain": fp64_ms,
                           "fp32_cv_with_training": cv_ms + 1e3 * train_s},
        # estimates after which training has paid for itself: training time / saving per estimate
        "break_even_estimates": (1e3 * train_s / saving) if saving > 0 else None,
        "estimate_median": {"fp32_cv": statistics.median(r.P for r in a),
                            "fp32_plain": statistics.median(r.P for r in b),
                            "fp64_plain": statistics.median(r.P for r in c)}}
    # the same trained networks at the benchmark's eps (the plain FP32 time there is the line's
    # time_to_eps_ms.asian)
    out["learned_cv"]["time_to_eps_ms_at_bench_eps"] = {
        "eps": EPS, "fp32_cv": statistics.median(
            mlmc.mlmc_estimate_cv(EPS, cv, s, Lmin=LMIN, Lmax=LMAX, N0=N0, stream=stream).wall_ms for s in seeds)}
    mlmc.mlmc_cv_free(cv)
    return out


def gpu_arm(args) -> None:
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1505_00965_gb300 import mlmc

    stream = torch.cuda.current_stream()
    seeds = rank_seeds(rank)
    problems = {p: mlmc.Problem(payoff=p, cash=1.0, **GBM) for p in PAYOFFS}

    def one_step():
        out = []
        for p in PAYOFFS:
            for s in seeds:
                out.append((p, mlmc.mlmc_estimate(EPS, problems[p], s, M=M, Lmin=LMIN, Lmax=LMAX, N0=N0,
                                                  precision="fp32", stream=stream)))
        return out

    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    # launch shapes: the autotuner's table (threads per block, lanes per path, samples per thread
    # and grid waves, measured per level and size class), made before the warm-up steps
    tuning = {"table": "planner"}
    if not args.no_autotune:
        import tempfile

        t = time.perf_counter()
        mlmc.mlmc_autotune_clear()
        for p in PAYOFFS:
            mlmc.mlmc_autotune(M=M, max_level=LMAX, precision="fp32", payoff=p, stream=stream)
        tuning = {"tune_s": time.perf_counter() - t, "entries": mlmc.mlmc_autotune_entries()}
        with tempfile.TemporaryDirectory() as tmp:
            path = os.path.join(tmp, "tuned.json")
            mlmc.mlmc_autotune_save(path)
            # one untimed step on each table, twice in turn (the faster of each kept)
            shape_ms = {"planner": [], "autotuned": []}
            for _ in range(2):
                for which in ("planner", "autotuned"):
                    mlmc.mlmc_autotune_clear()
                    if which == "autotuned":
                        mlmc.mlmc_autotune_load(path)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    one_step()
                    torch.cuda.synchronize()
                    shape_ms[which].append(1e3 * (time.perf_counter() - t0))
            tuning["step_ms"] = {k: min(v) for k, v in shape_ms.items()}
            # the timed steps run on the table that ran the untimed step faster
            mlmc.mlmc_autotune_clear()
            if tuning["step_ms"]["autotuned"] < tuning["step_ms"]["planner"]:
                mlmc.mlmc_autotune_load(path)
                tuning["table"] = "autotuned"
            else:
                tuning["table"] = "planner (the autotuned table ran the step slower)"
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid) if rank == 0 else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    dev_ms, wall_s, steps, instr, kern_ms, launches, d2h = 0.0, 0.0, 0.0, 0.0, 0.0, 0, 0
    tte = {p: [] for p in PAYOFFS}
    conv = {p: [] for p in PAYOFFS}
    last = None
    for _ in range(args.steps):
        flush.zero_()                     # L2 flushed between timed steps, outside their events
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t0 = time.perf_counter()
        res = one_step()
        t1 = time.perf_counter()
        e1.record(stream)
        torch.cuda.synchronize()
        dev_ms += e0.elapsed_time(e1)
        wall_s += t1 - t0
        for p, r in res:
            steps += r.path_steps
            instr += estimate_instructions(r.N, M, p)
            kern_ms += r.kernel_ms
            launches += r.launches
            d2h += r.d2h_bytes
            tte[p].append(r.wall_ms)
            conv[p].append(r.converged)
        last = res
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    dev_s, wall_max, steps_all, launches_all = combine_over_ranks(dev_ms / 1e3, wall_s, steps, float(launches))
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    sms = mlmc.mlmc_device_sm_count()
    run_mhz = (clocks or {}).get("sm_mhz") or None
    max_mhz = (clocks or {}).get("sm_max_mhz") or SM_MAX_MHZ_FALLBACK
    peak = sms * SCHEDULERS_PER_SM * WARP * max_mhz * 1e6 / 1e9          # G instructions / s
    achieved = instr / (kern_ms / 1e3) / 1e9
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Ginstr/s", "frac": achieved / peak,
                "traffic": TRAFFIC_BYTES_PER_LAUNCH, "traffic_basis": TRAFFIC_BASIS,
                "kernel": "level_ns2_kernel, level_kernel and level_small_kernel (FP32 paths, all levels of the "
                          "step; time = the driver's events around each "
                          "round on the engine stream, which bracket its four streams' launches)",
                "peak_basis": f"{sms} SMs x 4 schedulers x 32 lanes x {max_mhz:.0f} MHz (max SM clock), "
                              "one warp instruction per scheduler per clock",
                "frac_at_run_clock": (achieved / (sms * 128 * run_mhz * 1e6 / 1e9)) if run_mhz else None,
                "kernel_path_steps_per_s": steps / (kern_ms / 1e3)}
    # SFU: two hardware approximations per normal (log2 and sqrt per pair, sine and cosine per
    # pair), one normal per fine step, against the MUFU throughput the build's own probe measures
    probe = {}
    try:
        from paper_1505_00965_gb300 import peaks as peak_probe

        probe = peak_probe.measure()
        mufu = 2.0 * steps / (kern_ms / 1e3)
        roofline["sfu"] = {"achieved": mufu, "peak": probe["mufu_per_s"], "unit": "MUFU ops/s",
                           "frac": mufu / probe["mufu_per_s"],
                           "peak_basis": f"probe_peaks.cu: {probe['mufu_per_sm_per_clk']:.1f} MUFU ops per SM per clock"}
    except Exception as exc:  # the probe is a report; the benchmark line stands without it
        roofline["sfu"] = {"unavailable": str(exc)[:200]}

    # plain FP64 GPU MLMC on the same GPU, same eps (outside the timed region; Asian, the rank's
    # eight seeds, median as for FP32), and its kernels against the FP64 pipe's measured rate
    fp64_runs = [mlmc.mlmc_estimate(EPS, problems["asian"], s, M=M, Lmin=LMIN, Lmax=LMAX, N0=N0, precision="fp64",
                                    stream=stream) for s in seeds]
    fp64_ms = statistics.median(r.wall_ms for r in fp64_runs)
    fp32_asian_median = statistics.median(tte["asian"])
    fp64_steps = sum(r.path_steps for r in fp64_runs)
    fp64_kern_s = sum(r.kernel_ms for r in fp64_runs) / 1e3
    roofline_fp64 = {"bound": "fp64", "kernel": "level_kernel<double> and level_small_kernel<double> (FP64 paths, "
                                                "Asian, all levels of the eight estimates)",
                     "path_steps_per_s": fp64_steps / fp64_kern_s, "unit": "FP64 instructions/s",
                     "fp64_instructions_per_step": FP64_INSTR_PER_STEP, "fp64_instructions_basis": FP64_INSTR_BASIS}
    try:
        achieved64 = FP64_INSTR_PER_STEP * fp64_steps / fp64_kern_s
        roofline_fp64.update({"achieved": achieved64, "peak": probe["dfma_per_s"], "frac": achieved64 / probe["dfma_per_s"],
                              "peak_basis": f"probe_peaks.cu: {probe['dfma_per_sm_per_clk']:.3f} FP64 FMA per SM "
                                            "per clock (one FP64 instruction per operation)"})
    except Exception as exc:
        roofline_fp64["unavailable"] = str(exc)[:200]
    extras = {} if args.no_extras else side_workloads(mlmc, stream)
    value = steps_all / dev_s
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "eps": EPS, "payoffs": list(PAYOFFS), "M": M, "Lmax": LMAX, "N0": N0,
                   "seeds_per_gpu": SEEDS_PER_RANK, "precision": "FP32 paths, FP64 moment sums",
                   "l2": "512 MiB buffer written before every timed step, outside its events (the kernels read "
                         "no input arrays; they are compute bound)"},
        # the Asian estimates converge (bias test passed, MSE <= eps^2): time-to-eps
        "time_to_eps_ms": {"asian": fp32_asian_median},
        # the lookback estimates stop at L = Lmax with the bias test failing (discretely monitored
        # maximum, weak order 1/2): the time to run to Lmax and the bias left there
        "lookback_time_to_Lmax_ms": statistics.median(tte["lookback"]),
        "lookback_bias_estimate_at_Lmax": statistics.median(
            bias_estimate(r.mean, r.alpha) for q, r in last if q == "lookback"),
        "converged_fraction": {p: sum(v) / len(v) for p, v in conv.items()},
        "fp64_gpu_time_to_eps_ms": {"asian": fp64_ms, "seeds": "1..8 (median)"},
        "fp64_vs_fp32_time_to_eps": {"asian": fp64_ms / fp32_asian_median},
        "roofline_fp64": roofline_fp64,
        "estimates": {p: [r.P for q, r in last if q == p] for p in PAYOFFS},
        "gpu_launches": int(launches_all),
        "launch_shapes": tuning,
        "e2e": {"value": steps_all / wall_max, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": int(d2h / args.steps),
                "note": "mlmc_estimate through the C ABI: arguments by value (kernel parameters), results "
                        "copied device to host every round"},
        "roofline": roofline,
        "clocks": clocks,
    }
    line.update(extras)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(os.cpu_count() or 1)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------ one kernel on fixed arguments

def case_arm(args) -> None:
    """Launch one level kernel (or the control variate's lattice-mean kernel) on fixed
    arguments a few times and print its CUDA-event time per launch: the command that profiler
    captures of a single kernel run.  Not a benchmark line."""
    import torch

    from paper_1505_00965_gb300 import mlmc

    c = dict(kv.split("=", 1) for kv in args.case.split(",") if kv)
    level, m, n = int(c.get("level", 6)), int(c.get("M", 4)), int(float(c.get("N", 1e6)))
    reps, warm = int(c.get("reps", 3)), int(c.get("warmup", 1))
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if "train" in c:
        # the control variate's training launch: levels 0..train-1 of the Asian call
        prob = mlmc.Problem(payoff="asian", **GBM)
        for _ in range(max(reps, 1)):
            cv = mlmc.mlmc_cv_train(m, prob, seed=2024, levels=int(c["train"]), epochs=int(c.get("epochs", 20)),
                                    n_train=int(float(c.get("n_train", 1e6))), stream=stream)
            info = mlmc.mlmc_cv_train_info(cv)
            print(f"case {args.case}: training kernel {info['train_kernel_ms']:.3f} ms for {info['steps']} steps "
                  f"({1e3 * info['train_kernel_ms'] / max(info['steps'], 1):.2f} us per step), cluster "
                  f"{info['cluster']}, mlmc_cv_train {info['total_ms']:.1f} ms")
            mlmc.mlmc_cv_free(cv)
        return
    if "cv_level" in c:
        # the control-variate level kernel on a seeded random network (Asian call)
        import numpy as np

        lv = int(c["cv_level"])
        cv = mlmc.mlmc_cv_create(m, mlmc.Problem(payoff="asian", **GBM))
        theta = (np.random.default_rng(1).standard_normal(mlmc.MLMC_CV_PARAMS) * 0.2).astype(np.float32)
        mlmc.mlmc_cv_set_params(cv, lv, theta)
        d = torch.zeros(8, dtype=torch.float64, device="cuda")
        for _ in range(warm):
            mlmc.mlmc_cv_level_sums(cv, lv, n, 0, 1, d, stream=stream)
        e0.record(stream)
        for _ in range(reps):
            mlmc.mlmc_cv_level_sums(cv, lv, n, 0, 1, d, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / max(reps, 1)
        print(f"case {args.case}: {ms:.4f} ms per call (synchronising), {ms * 1e6 / n:.4f} ns per sample")
        mlmc.mlmc_cv_free(cv)
        return
    if "cv_mean" in c:
        import numpy as np

        R = int(c["cv_mean"])
        cv = mlmc.mlmc_cv_create(4, mlmc.Problem(payoff="asian"))
        theta = (np.random.default_rng(1).standard_normal(mlmc.MLMC_CV_PARAMS) * 0.2).astype(np.float32)
        mlmc.mlmc_cv_set_params(cv, 0, theta)
        d = torch.zeros(2, dtype=torch.float64, device="cuda")
        for _ in range(warm):
            mlmc.mlmc_cv_mean_sums(cv, 0, R, 0, 1, d, stream=stream)
        e0.record(stream)
        for _ in range(reps):
            mlmc.mlmc_cv_mean_sums(cv, 0, R, 0, 1, d, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / max(reps, 1)
        print(f"cv mean sample: {R} replicates, {ms:.4f} ms per launch, "
              f"{ms * 1e6 / (R * mlmc.MLMC_CV_LATTICE_POINTS):.4f} ns per lattice point")
        mlmc.mlmc_cv_free(cv)
        return
    prob = mlmc.Problem(payoff=c.get("payoff", "asian"), kind=c.get("kind", "gbm"), scheme=c.get("scheme", "em"))
    launch = {k: int(c[k]) for k in ("lanes_per_path", "threads_per_block", "blocks", "samples_per_thread") if k in c}
    precision = c.get("precision", "fp32")
    ws_bytes = mlmc.mlmc_level_workspace_bytes(level, m, n, precision, launch)
    ws = torch.zeros(ws_bytes, dtype=torch.uint8, device="cuda")
    d_sums = torch.zeros(4, dtype=torch.float64, device="cuda")

    def once():
        mlmc.mlmc_level_sums_async(level, m, n, 0, prob, 1, d_sums, ws, ws_bytes, precision=precision,
                                   launch=launch, stream=stream)

    for _ in range(warm):
        once()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        once()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(reps, 1)
    print(f"case {args.case}: {ms:.4f} ms/launch, {n * m ** level / ms / 1e9:.4g} T coupled steps/s, "
          f"sums={d_sums.tolist()}")


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batch and control-variate reports")
    ap.add_argument("--no-autotune", action="store_true", help="time the planner's launch shapes, not a tuned table")
    ap.add_argument("--case", default="", metavar="K=V,...",
                    help="time one kernel instead: level, M, N, payoff, kind, scheme, precision, "
                         "lanes_per_path, threads_per_block, blocks, samples_per_thread, reps, warmup; "
                         "or cv_mean=R (the lattice-mean kernel over R replicates)")
    args = ap.parse_args(argv)
    if args.case:
        case_arm(args)
        return
    if args.warmup < 3 and args.impl == "gb300":
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
