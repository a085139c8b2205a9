"""Measure the throughput of the units the level kernels use (MUFU, FP32 FMA, Philox4x32-10).

    python -m paper_1505_00965_gb300.peaks

Builds ``csrc/probe_peaks.cu`` into ``_build/probe_peaks`` (nvcc, sm_103a) and prints its JSON
line: operations per second and per SM per clock at the device's maximum clock.  The MUFU figure
is the SFU peak the benchmark's roofline compares the level kernels' two hardware
approximations per normal against.
"""
from __future__ import annotations

import json
import os
import subprocess

from .build import ARCH, BUILD_DIR, CSRC, NVCC


def build_probe() -> str:
    os.makedirs(BUILD_DIR, exist_ok=True)
    src = os.path.join(CSRC, "probe_peaks.cu")
    exe = os.path.join(BUILD_DIR, "probe_peaks")
    if not os.path.exists(exe) or os.path.getmtime(exe) < os.path.getmtime(src):
        subprocess.run([NVCC, *ARCH, "-O3", "-std=c++17", "-I", CSRC, "-o", exe, src], check=True)
    return exe


def measure() -> dict:
    out = subprocess.run([build_probe()], check=True, capture_output=True, text=True).stdout
    return json.loads(out.strip().splitlines()[-1])


def main() -> None:
    print(json.dumps(measure()))


if __name__ == "__main__":
    main()
