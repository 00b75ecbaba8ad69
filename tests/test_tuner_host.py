"""Host logic of the autotuner (choice, rounds, cache) with a fake timer: no GPU."""
import json

import pytest

import ucgen


@pytest.fixture(scope="module")
def mods():
    from paper_2607_03627_gb300 import binding, tune
    return binding, tune


def _fake_tuner(tune, times, cache_path):
    class FakeTuner(tune.Tuner):
        def __init__(self):
            super().__init__(cache_path=cache_path)
            self.calls = []

        @staticmethod
        def _gpu_name():
            return "fake GPU"

        def time_choice(self, ps, rpt, cta=0):
            self.calls.append((cta, rpt))
            t = times[(cta, rpt)]
            return t.pop(0) if isinstance(t, list) else t
    return FakeTuner()


def test_buckets_cover_every_size(mods):
    _, tune = mods
    assert tune.bucket_of(0) == 0
    for i, (lo, hi) in enumerate(tune.BUCKETS):
        assert tune.bucket_of(lo) == i and tune.bucket_of(hi - 1) == i
    assert tune.bucket_of(1 << 62) == len(tune.BUCKETS) - 1


def test_choose_takes_the_fastest_split_and_caches_it(mods, tmp_path):
    B, tune = mods
    ps = B.uc_presolve(B.uc_build_lp(ucgen.tiny(0)))
    path = str(tmp_path / "cache.json")
    t = _fake_tuner(tune, {(0, 1): 2.0, (0, 2): 1.5, (0, 4): 3.0}, path)
    assert t.choose(ps, 64) == 2
    assert sorted(r for _, r in t.calls) == [1, 2, 4]
    with open(path) as f:
        entry = json.load(f)[t.key(B.uc_presolved_dims(ps)[3], 64)]
    assert entry["rows_per_thread"] == 2
    again = _fake_tuner(tune, {}, path)          # a fresh tuner reads the cache, times nothing
    assert again.choose(ps, 64) == 2 and again.calls == []
    other = _fake_tuner(tune, {(0, 1): 1.0, (0, 2): 1.5, (0, 4): 3.0}, path)
    assert other.choose(ps, 32) == 1             # FP32 values: another cache key


def test_choose_pair_keeps_each_pairs_best_of_two_interleaved_rounds(mods, tmp_path):
    B, tune = mods
    ps = B.uc_presolve(B.uc_build_lp(ucgen.tiny(0)))
    times = {(128, 1): [1.0, 1.2], (128, 2): [1.3, 0.9], (256, 1): [1.1, 1.1], (256, 2): [1.4, 1.4]}
    t = _fake_tuner(tune, times, str(tmp_path / "cache.json"))
    assert t.choose_pair(ps, 64) == (128, 2)     # 0.9 in the second round beats 1.0 in the first
    order = [(128, 1), (128, 2), (256, 1), (256, 2)]
    assert t.calls == order + order              # interleaved, not one pair after another
    assert t.choose_pair(ps, 64) == (128, 2) and len(t.calls) == 8   # cached
