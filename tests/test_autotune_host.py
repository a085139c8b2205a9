"""The autotuner's table on the host: JSON round trip, size-class lookup, clearing (no GPU)."""
import os

import pytest


@pytest.fixture()
def mlmc():
    from paper_1505_00965_gb300 import build

    build.build()
    from paper_1505_00965_gb300 import mlmc as binding

    binding.mlmc_autotune_clear()
    yield binding
    binding.mlmc_autotune_clear()


def test_table_round_trip_and_lookup(mlmc, tmp_path):
    src = tmp_path / "tuned.json"
    src.write_text('{"entries": [\n'
                   ' {"precision": 1, "payoff": 1, "M": 4, "level": 6, "log2N": 10, "threads": 128, "lanes": 8, '
                   '"oversub": 1, "ns_per_sample": 12.5},\n'
                   ' {"precision": 1, "payoff": 1, "M": 4, "level": 6, "log2N": 19, "threads": 256, "lanes": 1, '
                   '"oversub": 2, "ns_per_sample": 3.25, "samples_per_thread": 2}\n'
                   ']}\n')
    assert mlmc.mlmc_autotune_load(str(src)) == 2
    assert mlmc.mlmc_autotune_entries() == 2
    # below the smallest class: the smallest class; between: the class below; above: the largest
    # (an entry without samples_per_thread, as older files wrote them, reads as one)
    assert mlmc.mlmc_autotune_lookup("fp32", "asian", 4, 6, 100) == (128, 8, 1, 1)
    assert mlmc.mlmc_autotune_lookup("fp32", "asian", 4, 6, 5000) == (128, 8, 1, 1)
    assert mlmc.mlmc_autotune_lookup("fp32", "asian", 4, 6, 1 << 19) == (256, 1, 2, 2)
    assert mlmc.mlmc_autotune_lookup("fp32", "asian", 4, 6, 1 << 30) == (256, 1, 2, 2)
    assert mlmc.mlmc_autotune_lookup("fp32", "asian", 4, 5, 1 << 19) is None
    assert mlmc.mlmc_autotune_lookup("fp64", "asian", 4, 6, 1 << 19) is None
    out = tmp_path / "again.json"
    mlmc.mlmc_autotune_save(str(out))
    mlmc.mlmc_autotune_clear()
    assert mlmc.mlmc_autotune_entries() == 0
    assert mlmc.mlmc_autotune_load(str(out)) == 2
    assert mlmc.mlmc_autotune_lookup("fp32", "asian", 4, 6, 1 << 20) == (256, 1, 2, 2)


def test_missing_file_is_an_error(mlmc, tmp_path):
    with pytest.raises(mlmc.MLMCError):
        mlmc.mlmc_autotune_load(str(tmp_path / "nope.json"))
