"""Philox4x32-10 evaluated by Triton's own `tl.philox` in interpreter mode (runs on the CPU).

Run as a child process (the interpreter switch must be set before Triton is imported):
reads a JSON list of [c0, c1, c2, c3, seed] from stdin, prints a JSON list of the four output
words for each.  Triton's seed maps to the key (seed low 32 bits, seed high 32 bits).
"""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(c_ptr, out_ptr, seed, BLOCK: tl.constexpr):
    i = tl.arange(0, BLOCK)
    c0 = tl.load(c_ptr + 4 * i + 0).to(tl.uint32, bitcast=True)
    c1 = tl.load(c_ptr + 4 * i + 1).to(tl.uint32, bitcast=True)
    c2 = tl.load(c_ptr + 4 * i + 2).to(tl.uint32, bitcast=True)
    c3 = tl.load(c_ptr + 4 * i + 3).to(tl.uint32, bitcast=True)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + 4 * i + 0, a.to(tl.int32, bitcast=True))
    tl.store(out_ptr + 4 * i + 1, b.to(tl.int32, bitcast=True))
    tl.store(out_ptr + 4 * i + 2, c.to(tl.int32, bitcast=True))
    tl.store(out_ptr + 4 * i + 3, d.to(tl.int32, bitcast=True))


def main():
    cases = json.load(sys.stdin)
    res = []
    for c0, c1, c2, c3, seed in cases:
        ctr = torch.tensor([c0, c1, c2, c3], dtype=torch.int64).to(torch.int32)
        out = torch.zeros(4, dtype=torch.int32)
        _philox_kernel[(1,)](ctr, out, seed, BLOCK=1)
        res.append([int(v) & 0xFFFFFFFF for v in out.tolist()])
    json.dump(res, sys.stdout)


if __name__ == "__main__":
    main()
