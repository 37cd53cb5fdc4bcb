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


class _P:
    def __init__(self, n, dim=2):
        self.n, self.dim = n, dim


class _FakeSampler:
    """Stands in for a BatchSampler: records the band thresholds it is set to."""

    def __init__(self, table):
        self.table, self.band, self.seen, self.closed = table, None, [], False

    def set_band_min_n(self, v):
        self.band = v
        self.seen.append(v)

    def set_coarse_threads(self, v):
        self.threads = v

    def close(self):
        self.closed = True


def test_cache_key_ignores_chain_order_and_counts_sizes():
    a = autotune.cache_key([_P(1023), _P(511), _P(1023)], "fp32")
    b = autotune.cache_key([_P(511), _P(1023), _P(1023)], "fp32")
    assert a == b == "2d|fp32|c=3|511x1,1023x2"
    assert autotune.cache_key([_P(1023)] * 3, "fp64") != a
    with pytest.raises(ValueError):
        autotune.cache_key([_P(7, 2), _P(7, 3)], "fp32")


def test_band_candidates_are_the_grids_between_coarse_and_finest():
    assert autotune.band_candidates([_P(1023)], 31) == [63, 127, 255, 511, autotune.TILES_ONLY]
    assert autotune.band_candidates([_P(255), _P(127)], 31) == [63, 127, autotune.TILES_ONLY]
    assert autotune.band_candidates([_P(63)], 31) == [autotune.TILES_ONLY]


def test_band_tuning_times_each_threshold_on_one_handle_and_keeps_the_best():
    table = {63: 1.10, 127: 1.02, 255: 0.98, 511: 1.01, autotune.TILES_ONLY: 1.05}
    s = _FakeSampler(table)
    best, ms = autotune.tune_band_min_n(s, table.keys(), timer=lambda smp: smp.table[smp.band])
    assert best == 255 and s.band == 255
    assert sorted(s.seen[:-1]) == sorted(table) and ms == table


def test_autotune_stores_the_fastest_pair_and_resolve_applies_it(tmp_path):
    path = tmp_path / "tune.json"
    ps = [_P(1023)] * 4
    # per coarse threshold a different landscape of band thresholds
    land = {15: {31: 2.2, 63: 2.0, 127: 1.9, 255: 1.8, 511: 1.85, autotune.TILES_ONLY: 2.1},
            31: {63: 1.2, 127: 1.1, 255: 1.0, 511: 1.05, autotune.TILES_ONLY: 1.3}}
    made = []

    def make(problems, c):
        s = _FakeSampler(land[c])
        made.append(s)
        return s

    # thread counts: 256 is 0.05 ms faster than the others
    def timer(smp):
        t = getattr(smp, "threads", None)
        return smp.table[smp.band] - (0.05 if t == 256 else 0.0)

    cache = autotune.TuneCache(str(path))
    out = autotune.autotune(ps, "fp32", coarse_candidates=(31, 15), cache=cache, make_sampler=make, timer=timer)
    assert (out["coarse_max_n"], out["band_min_n"], out["coarse_threads"]) == (31, 255, 256)
    assert all(s.closed for s in made) and len(out["ms"]) == 11 + 2 * len(autotune.COARSE_THREADS)
    # a fresh cache object reads the file back; explicit values win over it
    c2 = autotune.TuneCache(str(path))
    best = {"coarse_max_n": 31, "band_min_n": 255, "coarse_threads": 256}
    assert c2.get(autotune.cache_key(ps, "fp32")) == best
    assert autotune.resolve_settings(ps, "fp32", cache=c2) == best
    assert autotune.resolve_settings(ps, "fp32", band_min_n=0, cache=c2) == dict(best, band_min_n=0)
    assert autotune.resolve_settings(ps, "fp64", cache=c2) == autotune.DEFAULTS
    assert autotune.resolve_settings(ps, "fp32") == autotune.DEFAULTS


def test_cache_ignores_malformed_entries(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text('{"2d|fp32|c=1|7x1": {"coarse_max_n": -3}, "other": 5}')
    c = autotune.TuneCache(str(path))
    assert c.get("2d|fp32|c=1|7x1") is None and c.get("other") is None
    with pytest.raises(KeyError):
        c.put("k", {"tile": 3})
