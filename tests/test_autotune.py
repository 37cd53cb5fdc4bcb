"""Selection logic of the coarse-threshold autotuner (paper_2407_12149_gb300.autotune),
with the GPU timing replaced by a recorded table."""
import pytest

from paper_2407_12149_gb300 import autotune


def test_picks_the_fastest_candidate_and_times_each_once():
    calls = []

    def timer(ps, c):
        calls.append(c)
        return {15: 1.20, 31: 1.13, 63: 1.15}[c]

    best, t = autotune.autotune_coarse_max_n(["p"], candidates=(63, 31, 15, 31), timer=timer)
    assert best == 31
    assert sorted(calls) == [15, 31, 63]
    assert t == {15: 1.20, 31: 1.13, 63: 1.15}


def test_ties_go_to_the_smaller_threshold():
    assert autotune.pick_fastest({63: 1.0, 31: 1.0, 15: 2.0}) == 31


def test_rejects_empty_or_non_positive_candidates():
    with pytest.raises(ValueError):
        autotune.autotune_coarse_max_n(["p"], candidates=(), timer=lambda ps, c: 1.0)
    with pytest.raises(ValueError):
        autotune.autotune_coarse_max_n(["p"], candidates=(0, 31), timer=lambda ps, c: 1.0)
    with pytest.raises(ValueError):
        autotune.pick_fastest({})
