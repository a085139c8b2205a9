"""Host-side logic of bench.py on the CPU: seed sharding across ranks, the max-time / summed-work
reduction over ranks (two gloo processes), the instruction-count model and the clock parser."""
import os
import socket

import pytest

import bench


def test_rank_seeds_disjoint_and_first_rank_is_1_to_8():
    assert bench.rank_seeds(0) == list(range(1, 9))
    seen = set()
    for r in range(8):
        s = bench.rank_seeds(r)
        assert len(s) == 8 and not (seen & set(s))
        seen |= set(s)


def test_level_instruction_model():
    # level 0: a quarter Philox block, half a Box--Muller pair, one step, per-sample work
    assert bench.level_instructions(0, 4, "european") == 40 / 4 + 11 / 2 + 2 + 11
    # level l >= 1 with a running functional: 20 M^l + 11 ... plus the coarse terms
    nf = 4 ** 3
    want = 40 * nf / 4 + 11 * nf / 2 + 4 * nf + 2 * (nf // 4) + 11
    assert bench.level_instructions(3, 4, "asian") == want
    assert bench.estimate_instructions([10, 0, 2], 4, "european") == (
        10 * bench.level_instructions(0, 4, "european") + 2 * bench.level_instructions(2, 4, "european"))


def test_parse_clock_lines():
    lines = ["0, 1800, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Active",
             "0, 1900, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2000, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage"]
    c = bench.parse_clock_lines(lines)
    assert c["sm_mhz"] == 1900 and c["sm_max_mhz"] == 2070 and c["reasons"] == ["sw_power_cap"]
    assert bench.parse_clock_lines([])["sm_mhz"] is None


def test_clock_sampler_drops_its_start_up_sample(tmp_path, monkeypatch):
    """The sampler waits for nvidia-smi's first line before the timed region and drops it (here a
    stand-in script on PATH prints a 1000 MHz line first, then 2000 MHz lines)."""
    import time

    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '0, 1000, 2070, 100.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "while true; do\n"
                    "  echo '0, 2000, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "  sleep 0.05\n"
                    "done\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    sampler = bench.ClockSampler(None)
    time.sleep(0.3)
    c = sampler.stop()
    assert c["sm_mhz"] == 2000 and c["sm_max_mhz"] == 2070 and c["reasons"] == []


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    res = bench.combine_over_ranks(1.0 + rank, 10.0 - rank, 100.0 * (rank + 1), 7.0)
    out[rank] = res
    dist.destroy_process_group()


def test_combine_over_ranks_gloo_two_processes():
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        dev, wall, steps, launches = out[r]
        assert dev == 2.0 and wall == 10.0 and steps == 300.0 and launches == 14.0


def test_combine_without_group_is_identity():
    assert bench.combine_over_ranks(1.5, 2.5, 3.0, 4.0) == (1.5, 2.5, 3.0, 4.0)


def test_reference_arm_prints_one_line(monkeypatch, capsys):
    monkeypatch.setattr(bench, "ORACLE_SAMPLE", dict(eps=0.2, seeds=(1,)))
    monkeypatch.setenv("RANK", "0")
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    import json

    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == bench.UNIT
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert capsys.readouterr().out == ""
