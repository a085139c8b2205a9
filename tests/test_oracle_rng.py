"""Pins of the oracle's random input (the Brownian increments dW of Eq. (em), Sec. 2).

The stream is a reading (Philox4x32-10 + Box--Muller); it is pinned here against a library
implementation of Philox, against the exact uniform mapping, and against the normal law.
"""
import json
import os
import random
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def test_philox_matches_triton_interpreter():
    """Philox4x32-10 of random counters and keys equals Triton's `tl.philox` (interpreter, CPU)."""
    pytest.importorskip("triton")
    rng = random.Random(7)
    cases = [[0, 0, 0, 0, 0], [0xFFFFFFFF] * 4 + [2 ** 64 - 1]]
    cases += [[rng.getrandbits(32) for _ in range(4)] + [rng.getrandbits(64)] for _ in range(30)]
    proc = subprocess.run([sys.executable, os.path.join(HERE, "_triton_philox_ref.py")],
                          input=json.dumps(cases), capture_output=True, text=True, timeout=600)
    if proc.returncode != 0:
        pytest.skip("Triton interpreter unavailable: " + proc.stderr[-300:])
    ref = json.loads(proc.stdout)
    for case, want in zip(cases, ref):
        c0, c1, c2, c3, seed = case
        got = oracle.philox([c0, c1, c2, c3], [seed & 0xFFFFFFFF, seed >> 32])
        assert list(got) == want, case


def test_uniform_mapping_exact_endpoints():
    """Both uniform maps land in (0, 1] with the stated resolution."""
    assert oracle.uniform(0, "fp64") == 2.0 ** -32
    assert oracle.uniform(0xFFFFFFFF, "fp64") == 1.0
    assert oracle.uniform(0, "fp32") == 1.0
    assert oracle.uniform(0xFFFFFFFF, "fp32") == 2.0 ** -23
    assert oracle.uniform(0xFF400000, "fp32") == 0.5          # low 23 bits select 2^22
    assert oracle.uniform(0x00800000, "fp32") == 1.0          # bit 23 and above are unused
    assert oracle.uniform(0x7FFFFFFF, "fp64") == 0.5


def _many_normals(stream, n_samples=20000, level=3):
    z = [oracle.normals(11, level, s, 64, stream=stream) for s in range(n_samples // 64 + 1)]
    return np.concatenate(z)


@pytest.mark.parametrize("stream", ["fp64", "fp32"])
def test_normals_follow_standard_normal_law(stream):
    z = _many_normals(stream, 200_000)
    n = len(z)
    assert abs(z.mean()) < 4 / np.sqrt(n)
    assert abs(z.var() - 1) < 4 * np.sqrt(2 / n)
    assert abs(stats.kurtosis(z)) < 4 * np.sqrt(24 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_normals_independent_across_levels_tags_and_slots():
    n = 50_000
    a = np.concatenate([oracle.normals(3, 2, s, 16) for s in range(n // 16)])
    b = np.concatenate([oracle.normals(3, 3, s, 16) for s in range(n // 16)])
    c = np.concatenate([oracle.normals(3, 2, s, 16, tag=oracle.TAG_CV_MEAN) for s in range(n // 16)])
    d = np.concatenate([oracle.normals(4, 2, s, 16) for s in range(n // 16)])
    for x, y in [(a, b), (a, c), (a, d)]:
        assert abs(np.corrcoef(x, y)[0, 1]) < 4 / np.sqrt(len(x))
    # the two normals of one Box--Muller pair are uncorrelated
    assert abs(np.corrcoef(a[0::2], a[1::2])[0, 1]) < 4 / np.sqrt(len(a) / 2)
    # the same counter gives the same numbers
    assert np.array_equal(oracle.normals(3, 2, 5, 16), oracle.normals(3, 2, 5, 16))


def test_sample_normals_packing_rule():
    """Fine step k of a sample takes the sample's normal k; below four fine steps, 4 / M^l
    consecutive samples share one Philox block."""
    for s in [0, 1, 2, 3, 4, 17, 2 ** 33 + 5]:
        # level 0: four samples per block
        assert oracle.sample_normals(9, 0, 4, s)[0] == oracle.normals(9, 0, s // 4, 4)[s % 4]
        # level 1 with M = 2: two samples per block, two normals each
        np.testing.assert_array_equal(oracle.sample_normals(9, 1, 2, s),
                                      oracle.normals(9, 1, s // 2, 4)[2 * (s % 2):2 * (s % 2) + 2])
        # four or more fine steps: the sample's own blocks
        np.testing.assert_array_equal(oracle.sample_normals(9, 2, 4, s), oracle.normals(9, 2, s, 16))


def test_packed_level0_samples_independent():
    """Samples sharing a block (and a Box--Muller pair) are independent standard normals."""
    z = np.array([oracle.sample_normals(21, 0, 4, s)[0] for s in range(80_000)])
    n = len(z)
    for lag in (1, 2, 3, 4):
        assert abs(np.corrcoef(z[:-lag], z[lag:])[0, 1]) < 4.5 / np.sqrt(n)
    assert abs(z.mean()) < 4.5 / np.sqrt(n) and abs(z.var() - 1) < 4.5 * np.sqrt(2 / n)
